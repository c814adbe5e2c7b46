"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, derived from the arithmetic):
  * images: max-normalised error <= 1e-5 per (channel, product) -- FP32
    gridding, FP32 Stockham transforms (error ~ log2(N^2) * 2^-24 of max|E|),
    FP32 sums over <= 64 samples folded into FP64 accumulators;
  * gridded field: max |G_gpu - G_oracle| <= 2e-6 * max |G| (FP32 sums of a
    few dozen kernel products per cell);
  * F-stage spectra: <= 1e-5 of the stream's max |X|, and within 1e-4 of the
    oracle in scaled (code) units; 4-bit codes exact except where the
    oracle's scaled value is within 1e-4 of a rounding boundary, where one
    step either way is accepted (the FP32 and FP64 spectra may round apart
    only there).
Gains and kernels are handed to the oracle exactly as the library sees them
(rounded to complex64), so input quantisation is not counted as error.
"""
import os

import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IMG_TOL = 1e-5
GRID_TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def gpu_image(pos, taps, N, C, P, codes, gains, jones=False, scratch_mb=None, on_device=False):
    old = os.environ.get("MOFF_SCRATCH_MB")
    if scratch_mb is not None:
        os.environ["MOFF_SCRATCH_MB"] = str(scratch_mb)
    try:
        with moff.Plan(pos, taps, N, C, P, jones=jones) as pl:
            pl.set_gains(gains)
            if on_device:
                pl.submit(torch.from_numpy(np.ascontiguousarray(codes)).cuda())
            else:
                pl.submit(np.ascontiguousarray(codes))
            img, n = pl.read_image()
            info = pl.info()
    finally:
        if scratch_mb is not None:
            if old is None:
                os.environ.pop("MOFF_SCRATCH_MB", None)
            else:
                os.environ["MOFF_SCRATCH_MB"] = old
    return img, n, info


def random_case(seed, A, N, K, P, C, T, jones=False, spread=None):
    rng = np.random.default_rng(seed)
    spread = N if spread is None else spread
    pos = rng.uniform(0, spread, size=(A, 2)) + (N - spread) / 2
    if jones:
        taps = rng.normal(size=(A, 2, 2, K, K)) + 1j * rng.normal(size=(A, 2, 2, K, K))
    else:
        taps = rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K))
    re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    codes = synth.pack_4bit(re, im)
    gains = synth.gains_random(rng, C, A, P)
    return pos, c64(taps), codes, c64(gains)


def assert_image(img, ref, tol=IMG_TOL):
    err = oracle.max_norm_err(img, ref)
    assert err.max() <= tol, f"max-normalised error {err.max():.3e} > {tol:g} (per channel/product {err})"
    return err


# ------------------------------------------------------------------ gridding (Eq. m6 steps 1-2)

@pytest.mark.parametrize("N,P,K,A,jones", [(32, 1, 3, 64, False), (128, 2, 7, 300, False), (64, 2, 5, 40, True)])
def test_grid_snapshot_matches_oracle(N, P, K, A, jones):
    pos, taps, codes, gains = random_case(1, A, N, K, P, C=3, T=1, jones=jones)
    with moff.Plan(pos, taps, N, 3, P, jones=jones) as pl:
        pl.set_gains(gains)
        for chan in range(3):
            G = pl.grid_snapshot(np.ascontiguousarray(codes[0]), chan)
            W = oracle.grid_matrix(pos, taps, N, P, jones)
            y = oracle.calibrate(oracle.unpack_4bit(codes[0, chan]), gains[chan])
            ref = oracle.grid(y[None], W, N, P)[0]
            assert np.abs(G - ref).max() <= GRID_TOL * np.abs(ref).max()


# ------------------------------------------------------------------ whole image (Eq. m6)

def test_tiny_workload_image():
    """64 antennas, one pol, 16 channels, 256 samples, 32x32 grid, shared 3x3 kernel."""
    cfg = synth.config_tiny()
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    img, n, _ = gpu_image(cfg["pos"], taps, 32, 16, 1, cfg["codes"], gains)
    ref = oracle.moff_image(cfg["codes"], gains, cfg["pos"], taps, 32, 1)
    assert n == 256
    assert_image(img, ref)


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("P", [1, 2])
def test_image_every_grid_size(N, P):
    """Several stripes and column tiles, ragged time and channel chunks."""
    K = {32: 3, 64: 5, 128: 7, 256: 7, 512: 7}[N]
    A = {32: 50, 64: 120, 128: 400, 256: 600, 512: 900}[N]
    C, T = 3, 37
    pos, taps, codes, gains = random_case(10 + N + P, A, N, K, P, C, T)
    per = P * N * N * 8
    scratch = 2 * 7 * per / 2.0 ** 20               # MiB; forces chunks of a few samples
    img, n, info = gpu_image(pos, taps, N, C, P, codes, gains, scratch_mb=scratch)
    assert info["time_chunk"] < T
    ref = oracle.moff_image(codes, gains, pos, taps, N, P)
    assert_image(img, ref)


def test_image_jones_kernels():
    pos, taps, codes, gains = random_case(20, 60, 64, 5, 2, C=2, T=21, jones=True)
    img, _, _ = gpu_image(pos, taps, 64, 2, 2, codes, gains, jones=True)
    ref = oracle.moff_image(codes, gains, pos, taps, 64, 2, jones=True)
    assert_image(img, ref)


def test_dense_core_global_contribution_lists():
    """So many antennas per grid row that the kernel lists stay in global memory."""
    rng = np.random.default_rng(21)
    N, K, A = 64, 15, 1500
    pos = rng.uniform(0, N, size=(A, 2))
    taps = c64(rng.normal(size=(A, 1, K, K)) + 1j * rng.normal(size=(A, 1, K, K)))
    codes = synth.pack_4bit(rng.integers(-7, 8, size=(5, 1, A, 1)), rng.integers(-7, 8, size=(5, 1, A, 1)))
    gains = c64(synth.gains_random(rng, 1, A, 1))
    img, _, _ = gpu_image(pos, taps, N, 1, 1, codes, gains)
    ref = oracle.moff_image(codes, gains, pos, taps, N, 1)
    assert_image(img, ref)


# ------------------------------------------------------------------ edge cases

def test_single_antenna_wrapping_footprint_and_delta_kernel():
    N = 32
    pos = np.array([[31.7, 0.2]])          # anchor (32 -> 0, 0): footprint wraps both axes
    rng = np.random.default_rng(30)
    taps = c64(rng.normal(size=(1, 1, 5, 5)) + 1j * rng.normal(size=(1, 1, 5, 5)))
    codes = synth.pack_4bit(rng.integers(-8, 8, size=(3, 1, 1, 1)), rng.integers(-8, 8, size=(3, 1, 1, 1)))
    gains = c64(np.array([[[0.7 - 0.2j]]]))
    img, _, _ = gpu_image(pos, taps, N, 1, 1, codes, gains)
    assert_image(img, oracle.moff_image(codes, gains, pos, taps, N, 1))
    # delta kernel: the image is flat and equals sum_t |g x|^2
    img1, _, _ = gpu_image(pos, np.ones((1, 1, 1, 1)), N, 1, 1, codes, gains)
    flat = np.sum(np.abs(oracle.unpack_4bit(codes[:, 0, 0, 0]) * gains[0, 0, 0]) ** 2)
    np.testing.assert_allclose(img1[0, 0], np.full((N, N), flat), rtol=1e-6)


def test_zero_voltages_give_zero_and_one_sample_works():
    pos, taps, codes, gains = random_case(31, 30, 64, 3, 2, C=2, T=1)
    img, n, _ = gpu_image(pos, taps, 64, 2, 2, np.zeros_like(codes), gains)
    assert n == 1 and np.all(img == 0)
    img, _, _ = gpu_image(pos, taps, 64, 2, 2, codes, gains)
    assert_image(img, oracle.moff_image(codes, gains, pos, taps, 64, 2))


def test_accumulation_across_blocks_reset_and_device_input():
    pos, taps, codes, gains = random_case(32, 80, 64, 5, 2, C=3, T=30)
    ref = oracle.moff_image(codes, gains, pos, taps, 64, 2)
    with moff.Plan(pos, taps, 64, 3, 2) as pl:
        pl.set_gains(gains)
        pl.submit(np.ascontiguousarray(codes[:11]))
        pl.submit(torch.from_numpy(np.ascontiguousarray(codes[11:]).copy()).cuda())
        img, n = pl.read_image(reset=True)
        assert n == 30
        assert_image(img, ref)
        img2, n2 = pl.read_image()
        assert n2 == 0 and np.all(img2 == 0)
        # device output buffer
        pl.submit(np.ascontiguousarray(codes))
        out = torch.empty((3, 4, 64, 64), dtype=torch.float32, device="cuda")
        pl.read_image(out=out)
        assert_image(out.cpu().numpy(), ref)


def test_bitwise_deterministic_repeat():
    pos, taps, codes, gains = random_case(33, 200, 128, 7, 2, C=2, T=9)
    a, _, _ = gpu_image(pos, taps, 128, 2, 2, codes, gains)
    b, _, _ = gpu_image(pos, taps, 128, 2, 2, codes, gains, on_device=True)
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ full-size dual-pol array, sampled channels

def test_dualpol_full_size_sampled_channels():
    """1024-antenna hex core, 128x128 grid, 7x7 complex kernels, 1024 channels,
    1000 samples -- the launch configuration of the benchmark -- checked on
    three sampled channels against the oracle."""
    cfg = synth.config_dualpol()
    T, C, A, P, N = 1000, cfg["n_chan"], cfg["pos"].shape[0], 2, cfg["grid_n"]
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    codes_d = synth.device_codes(8123669 + 101, T, C, A, P)
    with moff.Plan(cfg["pos"], taps, N, C, P) as pl:
        pl.set_gains(gains)
        pl.submit(codes_d)
        img, n = pl.read_image()
    assert n == T
    chans = [0, 517, 1023]
    sub = codes_d[:, chans].cpu().numpy()
    ref = oracle.moff_image(sub, gains[chans], cfg["pos"], taps, N, P)
    assert_image(img[chans], ref)


def test_filled_aperture_full_array_sampled():
    """The precision configuration's array at full size -- 16384 antennas filling
    a 128 x 128 lambda lattice, dual pol, 7x7 kernels, 512 x 512 grid -- on the FP32
    path, 4 channels x 24 samples against the oracle.  The FP16 tensor-core path
    takes this density by the factored-DFT route (more than 128 antennas' kernel
    rows land on a grid row, too many for the row-spectrum contraction), within
    the reduced-precision bar."""
    cfg = synth.config_precision(n_chan=4)
    T, C, A, P, N = 24, 4, cfg["pos"].shape[0], 2, cfg["grid_n"]
    assert A == 16384 and N == 512
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    codes_d = synth.device_codes(8123669 + 102, T, C, A, P)
    with moff.Plan(cfg["pos"], taps, N, C, P) as pl:
        pl.set_gains(gains)
        pl.submit(codes_d)
        img, n = pl.read_image()
    assert n == T
    ref = oracle.moff_image(codes_d.cpu().numpy(), gains, cfg["pos"], taps, N, P)
    assert_image(img, ref)
    with moff.Plan(cfg["pos"], taps, N, C, P, fp16tc=True) as pl:
        assert pl.route() in ("fp16_dft", "fp16_tcgrid")
        pl.set_gains(gains)
        pl.submit(codes_d)
        img16, n = pl.read_image()
    err = oracle.max_norm_err(img16, ref)
    print("filled aperture, FP16 factored-DFT route: max-normalised error per image",
          " ".join(f"{e:.2e}" for e in err.max(axis=1)))
    assert n == T and err.max() <= 3e-3


def test_widefield_full_array_sampled():
    """The wide-field configuration's array at full size -- 32768 antennas on a
    256 x 128 lambda lattice (x wraps the 512-cell grid), 9x9 Jones kernels with a
    w-phase -- on 2 channels x 6 samples against the oracle."""
    cfg = synth.config_widefield(n_chan=2)
    T, C, A, P, N = 6, 2, cfg["pos"].shape[0], 2, cfg["grid_n"]
    assert A == 32768 and N == 512 and cfg["taps"].shape == (A, 2, 2, 9, 9)
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    codes_d = synth.device_codes(8123669 + 104, T, C, A, P)
    with moff.Plan(cfg["pos"], taps, N, C, P, jones=True) as pl:
        pl.set_gains(gains)
        pl.submit(codes_d)
        img, n = pl.read_image()
    assert n == T
    ref = oracle.moff_image(codes_d.cpu().numpy(), gains, cfg["pos"], taps, N, P, jones=True)
    assert_image(img, ref)


# ------------------------------------------------------------------ F-stage (Eq. FFTofE)

def _pfb_case(seed, A, P, C, ntaps, F):
    rng = np.random.default_rng(seed)
    M = 2 * C
    adc = synth.adc_stream(rng, A, P, (F + ntaps - 1) * M, sigma=20.0,
                           tones=[(5.0 / M, 30.0), ((C // 3 + 0.25) / M, 25.0)])
    return adc


@pytest.mark.parametrize("C,ntaps,A,P,F", [(32, 4, 5, 2, 9), (256, 8, 3, 2, 5), (1024, 8, 17, 2, 4), (1024, 8, 3, 2, 70),
                                           (1024, 4, 2, 1, 5), (2048, 8, 2, 1, 3)])
def test_fstage_spectra_and_codes(C, ntaps, A, P, F):
    adc = _pfb_case(40 + C, A, P, C, ntaps, F)
    M = 2 * C
    h = oracle.pfb_window(ntaps, M).astype(np.float32).astype(np.float64)
    X = oracle.pfb_spectra(adc, h, ntaps, M)                           # [A, P, F, C]
    Xr = np.transpose(X, (2, 3, 0, 1))                                  # [F, C, A, P]
    scale = 2.0 / np.std(np.abs(X))
    pos = np.zeros((A, 2))
    with moff.Plan(pos, np.ones((A, P, 1, 1)), 32, C, P, fstage=True) as pl:
        pl.set_fstage(ntaps, None, scale)
        spec = pl.channelise(adc, kind=1)
        codes = pl.channelise(adc, kind=0)
        pl.set_fstage(ntaps, h.astype(np.float32), scale)
        codes2 = pl.channelise(adc, kind=0)
    den = np.abs(Xr).max(axis=(0, 1))
    assert (np.abs(spec - Xr).max(axis=(0, 1)) <= 1e-5 * den).all()
    # the band below must cover the FP32-FP64 difference in the units the rounding sees
    d_scaled = float(np.abs(spec - Xr).max()) * float(np.float32(scale))
    print(f"C={C} taps={ntaps}: max FP32-FP64 spectrum difference {d_scaled:.2e} codes")
    assert d_scaled < 1e-4
    re, im = oracle.quantise_4bit(Xr, np.float32(scale))
    z = oracle.unpack_4bit(codes)
    amb = oracle.ambiguous_codes(Xr, np.float32(scale), 1e-4)
    dr, di = np.abs(z.real - re), np.abs(z.imag - im)
    assert (dr[~amb] == 0).all() and (di[~amb] == 0).all()
    assert dr.max() <= 1 and di.max() <= 1
    assert np.array_equal(codes, codes2)


def test_adc_to_image_end_to_end():
    """ADC -> F-stage -> image.  The seed is the first one (from a fixed start)
    whose oracle spectra have no component within 2e-5 (scaled units; the FP32
    spectra differ from FP64 by ~2e-6 there) of a rounding boundary, so the
    4-bit codes are unique and the image must match to the FP32 bar."""
    A, P, C, ntaps, F, N = 8, 2, 32, 4, 8, 32
    M = 2 * C
    h = oracle.pfb_window(ntaps, M).astype(np.float32).astype(np.float64)
    for seed in range(500, 700):
        adc = _pfb_case(seed, A, P, C, ntaps, F)
        X = oracle.pfb_spectra(adc, h, ntaps, M)
        scale = np.float32(2.0 / np.std(np.concatenate([X.real.ravel(), X.imag.ravel()])))
        if not oracle.ambiguous_codes(X, scale, 2e-5).any():
            break
    else:
        pytest.skip("no boundary-free seed in range")
    codes_ref, _ = oracle.channelise(adc, h, ntaps, M, scale)
    rng = np.random.default_rng(seed)
    pos = rng.uniform(4, 28, size=(A, 2))
    taps = c64(rng.normal(size=(A, P, 3, 3)) + 1j * rng.normal(size=(A, P, 3, 3)))
    gains = c64(synth.gains_random(rng, C, A, P))
    with moff.Plan(pos, taps, N, C, P, fstage=True) as pl:
        pl.set_fstage(ntaps, None, float(scale))
        pl.set_gains(gains)
        pl.submit_adc(adc)
        img, n = pl.read_image()
    assert n == F
    ref = oracle.moff_image(codes_ref, gains, pos, taps, N, P)
    assert_image(img, ref)


# ------------------------------------------------------------------ errors and fault injection (host side)

def test_state_and_argument_errors_on_gpu():
    pos, taps, codes, gains = random_case(50, 10, 32, 3, 1, C=2, T=2)
    with moff.Plan(pos, taps, 32, 2, 1) as pl:
        with pytest.raises(moff.MoffError) as e:
            pl.submit_adc(np.zeros((10, 1, 4096), np.int8))
        assert e.value.status == -4
        with pytest.raises(moff.MoffError) as e:
            moff.moff_submit(pl.handle, np.zeros((0, 2, 10, 1), np.uint8))
        assert e.value.status == -1
        with pytest.raises(moff.MoffError):
            pl.grid_snapshot(np.ascontiguousarray(codes[0]), 5)
    with moff.Plan(pos, taps, 32, 64, 1, fstage=True) as pl:
        with pytest.raises(moff.MoffError) as e:
            pl.submit_adc(np.zeros((10, 1, 1000), np.int8))      # not a multiple of M
        assert e.value.status == -1
        with pytest.raises(moff.MoffError) as e:
            pl.submit_adc(np.zeros((10, 1, 128 * 3), np.int8))   # shorter than the filter
        assert e.value.status == -1


def test_allocation_failure_is_reported_and_recoverable():
    import subprocess
    import sys
    code = (
        "import numpy as np, paper_0812_3669_gb300 as m\n"
        "pos=np.zeros((4,2)); taps=np.ones((4,1,3,3))\n"
        "try:\n    m.Plan(pos,taps,32,2,1)\n    print('NOFAIL')\n"
        "except m.MoffError as e:\n    print('STATUS', e.status)\n"
        "p=m.Plan(pos,taps,32,2,1); p.submit(np.zeros((2,2,4,1),np.uint8)); img,n=p.read_image(); print('OK', n)\n"
    )
    env = dict(os.environ, MOFF_FAULT="alloc:3")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert "STATUS -2" in r.stdout, r.stdout + r.stderr
    assert "OK 2" in r.stdout, r.stdout + r.stderr


def test_adc_path_equals_channelise_then_submit():
    """submit_adc is the F-stage followed by the imaging path: its image equals,
    bit for bit, submitting the library's own channelised codes."""
    A, P, C, ntaps, F, N = 30, 2, 128, 8, 12, 64
    adc = _pfb_case(77, A, P, C, ntaps, F)
    rng = np.random.default_rng(78)
    pos = rng.uniform(8, 56, size=(A, 2))
    taps = c64(rng.normal(size=(A, P, 5, 5)) + 1j * rng.normal(size=(A, P, 5, 5)))
    gains = c64(synth.gains_random(rng, C, A, P))
    with moff.Plan(pos, taps, N, C, P, fstage=True) as pl:
        pl.set_fstage(ntaps, None, 0.07)
        pl.set_gains(gains)
        pl.submit_adc(adc)
        a, n1 = pl.read_image(reset=True)
        codes = pl.channelise(adc, kind=0)
        pl.submit(codes)
        b, n2 = pl.read_image(reset=True)
    assert n1 == n2 == F
    assert np.array_equal(a, b)


# ------------------------------------------------------------------ gridding shapes

@pytest.mark.parametrize("N,P,K,A,jones,stage", [(64, 2, 5, 150, False, "0"), (128, 2, 7, 300, False, "1"),
                                                  (64, 2, 5, 40, True, "0"), (256, 1, 3, 200, False, "1"),
                                                  (32, 1, 3, 64, False, "0")])
def test_cell_pair_and_block_lanes_are_bit_identical(monkeypatch, N, P, K, A, jones, stage):
    """Pair lanes and 2 x 2 block lanes sum each cell's contributions in the
    single-cell order (plus exact zero terms), so the images and the gridded
    snapshot must match the single-cell kernel bit for bit, with entries read
    through L2 or staged (blocks always read them through L2)."""
    pos, taps, codes, gains = random_case(500 + N, A, N, K, P, C=3, T=21, jones=jones)
    monkeypatch.setenv("MOFF_GRID_STAGE", stage)
    out = {}
    for cpl, pairs, quads in ((1, "0", "0"), (2, "1", "0"), (4, "1", "1")):
        monkeypatch.setenv("MOFF_GRID_PAIRS", pairs)
        monkeypatch.setenv("MOFF_GRID_QUADS", quads)
        with moff.Plan(pos, taps, N, 3, P, jones=jones) as pl:
            assert pl.tuning()["cells_per_lane"] == cpl
            pl.set_gains(gains)
            pl.submit(codes)
            img, n = pl.read_image()
            snap = pl.grid_snapshot(codes[4], 1)
        out[cpl] = (img, snap)
    for cpl in (2, 4):
        assert np.array_equal(out[1][0], out[cpl][0])
        assert np.array_equal(out[1][1], out[cpl][1])
    assert_image(out[4][0], oracle.moff_image(codes, gains, pos, taps, N, P, jones=jones))


@pytest.mark.parametrize("N,P,K,A", [(32, 1, 3, 60), (64, 2, 5, 150), (128, 2, 7, 300), (256, 2, 5, 250),
                                     (512, 1, 3, 120)])
def test_wide_stripes_and_in_place_row_passes_are_bit_identical(monkeypatch, N, P, K, A):
    """Stripes of twice the rows (wide) run the first row-transform pass in place
    where each lane holds one slot (N = 32, 128, 256 wide; N = 64 plain), with one
    row buffer and capped registers; the other shapes keep two buffers.  The
    per-cell sums and the per-row passes are the same arithmetic in every shape,
    so every (wide, lanes) combination must give the same image and gridded
    snapshot bit for bit, and match the oracle."""
    C, T = 2, 19                     # T not a multiple of the samples per pass
    pos, taps, codes, gains = random_case(900 + N, A, N, K, P, C=C, T=T)
    monkeypatch.setenv("MOFF_GRID_STAGE", "0")
    out = {}
    for wide in ("0", "1"):
        for cpl, pairs, quads in ((1, "0", "0"), (2, "1", "0"), (4, "1", "1")):
            monkeypatch.setenv("MOFF_GRID_WIDE", wide)
            monkeypatch.setenv("MOFF_GRID_PAIRS", pairs)
            monkeypatch.setenv("MOFF_GRID_QUADS", quads)
            try:
                pl = moff.Plan(pos, taps, N, C, P)
            except moff.MoffError:
                assert cpl == 4              # 2 x 2 blocks need an even stripe height
                continue
            with pl:
                tu = pl.tuning()
                assert (tu["cells_per_lane"], tu["wide_rows"]) == (cpl, int(wide))
                pl.set_gains(gains)
                pl.submit(codes)
                img, n = pl.read_image()
                snap = pl.grid_snapshot(codes[3], 1)
            assert n == T
            out[(wide, cpl)] = (img, snap)
    assert ("0", 1) in out and ("1", 1) in out and len(out) >= 4
    base = out[("0", 1)]
    for key, (img, snap) in out.items():
        assert np.array_equal(img, base[0]), key
        assert np.array_equal(snap, base[1]), key
    assert_image(base[0], oracle.moff_image(codes, gains, pos, taps, N, P))


def test_host_adc_pipelined_staging_equals_device_input():
    """A host ADC block longer than one staging segment (128 frames) is copied in
    frame segments that overlap the F-stage and imaging of earlier ones; the
    result (image, F-stage frames, beams) must equal the device-input submit."""
    A, P, C, N, ntaps, F = 6, 2, 64, 32, 8, 300
    rng = np.random.default_rng(77)
    pos = rng.uniform(4, 28, size=(A, 2))
    taps = c64(rng.normal(size=(A, P, 3, 3)) + 1j * rng.normal(size=(A, P, 3, 3)))
    adc = synth.adc_stream(rng, A, P, (F + ntaps - 1) * 2 * C, sigma=20.0)
    out = []
    for host in (True, False):
        with moff.Plan(pos, taps, N, C, P, fstage=True) as pl:
            pl.set_fstage(ntaps, None, 0.03)
            pl.set_beams([3, 17], [5, 30])
            src = adc if host else torch.from_numpy(adc).cuda()
            pl.submit_adc(src)
            beams = pl.read_beams()
            img, n = pl.read_image()
        assert n == F and beams.shape == (F, C, 2, P)
        out.append((img, beams))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
