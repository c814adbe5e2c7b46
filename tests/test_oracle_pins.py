"""Pins of the FP64 oracle against things other than itself (CPU only).

Every function of ``oracle`` is checked here against hand-worked fixtures
(tests/golden), closed forms, textbook special cases, library routines or an
independent formulation (the FX route of Eqs. visDef/Bdef/RBeamEq), chosen so
that a dropped term, a sign error or a transposed operand fails a test.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def _codes_from_complex(z):
    z = np.asarray(z)
    return synth.pack_4bit(np.rint(z.real).astype(int), np.rint(z.imag).astype(int))


# ------------------------------------------------------------------ unpack / anchors / quantise

def test_unpack_golden():
    rows = read_golden("unpack_4bit.txt")
    codes = np.array([int(r[0], 16) for r in rows], dtype=np.uint8)
    want = np.array([int(r[1]) + 1j * int(r[2]) for r in rows])
    np.testing.assert_array_equal(oracle.unpack_4bit(codes), want)


def test_unpack_is_inverse_of_pack_over_all_256_codes():
    re, im = np.meshgrid(np.arange(-8, 8), np.arange(-8, 8), indexing="ij")
    codes = synth.pack_4bit(re.ravel(), im.ravel())
    assert len(set(codes.tolist())) == 256
    z = oracle.unpack_4bit(codes)
    np.testing.assert_array_equal(z.real, re.ravel())
    np.testing.assert_array_equal(z.imag, im.ravel())


def test_anchor_golden():
    rows = read_golden("anchors.txt")
    pos = np.array([[float(r[0]), float(r[1])] for r in rows])
    want = np.array([[int(r[2]), int(r[3])] for r in rows])
    np.testing.assert_array_equal(oracle.anchors(pos), want)


def test_quantise_golden():
    rows = read_golden("quantise_4bit.txt")
    v = np.array([float(r[0]) for r in rows])
    want = np.array([int(r[1]) for r in rows])
    re, im = oracle.quantise_4bit(v + 1j * v[::-1], 1.0)
    np.testing.assert_array_equal(re, want)
    np.testing.assert_array_equal(im, want[::-1])
    re2, _ = oracle.quantise_4bit(v / 4.0, 4.0)
    np.testing.assert_array_equal(re2, want)


def test_ambiguous_mask():
    v = np.array([0.5 + 1e-7, 0.3, 6.5 - 2e-7, 7.5, -7.5, -6.5 + 1e-8, 2.0])
    m = oracle.ambiguous_codes(v, 1.0, 1e-6)
    np.testing.assert_array_equal(m, [True, False, True, False, False, True, False])


# ------------------------------------------------------------------ transform

def test_sky_transform_equals_naive_dft():
    rng = np.random.default_rng(1)
    N = 8
    G = rng.normal(size=(2, N, N)) + 1j * rng.normal(size=(2, N, N))
    E = oracle.sky_transform(G)
    want = np.zeros_like(G)
    for ky in range(N):
        for kx in range(N):
            for ry in range(N):
                for rx in range(N):
                    want[:, ky, kx] += G[:, ry, rx] * np.exp(2j * np.pi * (ky * ry + kx * rx) / N)
    np.testing.assert_allclose(E, want, rtol=0, atol=1e-11)


# ------------------------------------------------------------------ closed forms

def _integer_layout(rng, A, N, spacing):
    """A antennas at distinct integer cells, at least ``spacing`` apart in x or y."""
    cells = []
    while len(cells) < A:
        c = rng.integers(0, N, size=2)
        if all(max(abs(int(c[0]) - a), abs(int(c[1]) - b)) >= spacing for a, b in cells):
            cells.append((int(c[0]), int(c[1])))
    return np.array(cells, dtype=np.float64)


def test_point_source_closed_form_and_sign():
    """Delta kernels, unit gains, one noiseless source at theta_s = (kx, ky) = (0, 8)
    with amplitude 7: the image is 49 T |sum_a exp(+2 pi i p_a.(k - theta_s)/N)|^2,
    peaking at +theta_s with 49 T A^2 (pins the transform's sign, Eq. Ea vs Eq. m6)."""
    rng = np.random.default_rng(2)
    N, A, T = 32, 20, 5
    pos = _integer_layout(rng, A, N, 1)
    th = np.array([0, 8])
    x = 7 * np.exp(-2j * np.pi * (pos @ th) / N)              # in {+-7, +-7i}
    codes = np.broadcast_to(_codes_from_complex(x)[None, None, :, None], (T, 1, A, 1)).copy()
    taps = np.ones((A, 1, 1, 1), dtype=complex)
    gains = np.ones((1, A, 1), dtype=complex)
    I = oracle.moff_image(codes, gains, pos, taps, N, 1)[0, 0]
    k = np.stack(np.meshgrid(np.arange(N), np.arange(N), indexing="xy"), axis=-1)  # [ky][kx] -> (kx, ky)
    phase = np.exp(2j * np.pi * np.einsum("yxc,ac->yxa", k - th, pos) / N)
    want = 49 * T * np.abs(phase.sum(axis=-1)) ** 2
    np.testing.assert_allclose(I, want, rtol=1e-12, atol=1e-9)
    assert np.unravel_index(np.argmax(I), I.shape) == (th[1], th[0])
    assert abs(I[th[1], th[0]] - 49 * T * A * A) < 1e-6


def test_frequency_scaled_positions_keep_the_source_pixel():
    """Channel-dependent positions (Sec. 4 names frequency-dependent imaging effects;
    uv positions in wavelengths scale with frequency): channel c sees the array at
    s_c times its reference positions.  A source at theta_s observed with each
    channel's own positions peaks at +theta_s in every channel with 49 T A^2 and the
    closed-form PSF of that channel's positions; a set mix-up would misplace it."""
    rng = np.random.default_rng(21)
    N, A, T = 32, 12, 3
    base = _integer_layout(rng, A, N // 3, 1)                       # 0..10, so 3x stays on the grid
    scale = [1, 2, 3, 2]                                            # chan_group = [0, 1, 2, 1]
    sets = np.stack([base * s for s in (1, 2, 3)])
    grp = [0, 1, 2, 1]
    th = np.array([8, 16])
    codes = np.zeros((T, len(grp), A, 1), dtype=np.uint8)
    for c, g in enumerate(grp):
        x = 7 * np.exp(-2j * np.pi * (sets[g] @ th) / N)           # in {+-7, +-7i}
        codes[:, c, :, 0] = _codes_from_complex(x)[None]
    taps = np.ones((3, A, 1, 1, 1), dtype=complex)
    gains = np.ones((len(grp), A, 1), dtype=complex)
    I = oracle.moff_image_sets(codes, gains, sets, taps, grp, N, 1)
    k = np.stack(np.meshgrid(np.arange(N), np.arange(N), indexing="xy"), axis=-1)
    for c, g in enumerate(grp):
        phase = np.exp(2j * np.pi * np.einsum("yxc,ac->yxa", k - th, sets[g]) / N)
        np.testing.assert_allclose(I[c, 0], 49 * T * np.abs(phase.sum(axis=-1)) ** 2, rtol=1e-12, atol=1e-9)
        assert abs(I[c, 0, th[1], th[0]] - 49 * T * A * A) < 1e-6
    assert scale[3] == scale[1] and np.array_equal(I[1], I[3])
    # one set for every channel is the plain image
    one = oracle.moff_image_sets(codes, gains, sets[:1], taps[:1], [0] * len(grp), N, 1)
    np.testing.assert_array_equal(one, oracle.moff_image(codes, gains, sets[0], taps[0], N, 1))


def test_edge_padding_samples_the_same_image():
    """Image oversampling by edge padding of the FFT input (Sec. 4): with footprints
    that wrap on neither grid, the image on a 2N grid at even pixels equals the
    N-grid image (a DFT of a zero-padded field, sampled at every second frequency)."""
    rng = np.random.default_rng(22)
    N, A, T, K, P = 16, 7, 4, 3, 2
    pos = rng.uniform(2, N - 3, size=(A, 2))
    taps = rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K))
    codes = _codes_from_complex(rng.integers(-7, 8, size=(T, 1, A, P)) + 1j * rng.integers(-7, 8, size=(T, 1, A, P)))
    gains = np.exp(1j * rng.uniform(0, 6, size=(1, A, P)))
    I1 = oracle.moff_image(codes, gains, pos, taps, N, P)
    I2 = oracle.moff_image(codes, gains, pos, taps, 2 * N, P)
    np.testing.assert_allclose(I2[:, :, ::2, ::2], I1, rtol=0, atol=1e-9 * np.abs(I1).max())
    assert np.abs(I2[:, :2, 1::2, 1::2]).max() > 0          # the padded grid adds the in-between pixels


def test_shared_kernel_multiplies_by_kernel_power():
    """A kernel shared by every antenna multiplies the delta-kernel image by |K^(k)|^2,
    K^(k) = sum_d t[d] exp(+2 pi i k.(d - K//2)/N)."""
    rng = np.random.default_rng(3)
    N, A, T, K = 16, 9, 4, 3
    pos = _integer_layout(rng, A, N, 1)
    t = rng.normal(size=(K, K)) + 1j * rng.normal(size=(K, K))
    codes = _codes_from_complex(rng.integers(-7, 8, size=(T, 1, A, 1)) + 1j * rng.integers(-7, 8, size=(T, 1, A, 1)))
    gains = np.exp(1j * rng.uniform(0, 6, size=(1, A, 1)))
    I_k = oracle.moff_image(codes, gains, pos, np.broadcast_to(t, (A, 1, K, K)), N, 1)[0, 0]
    I_d = oracle.moff_image(codes, gains, pos, np.ones((A, 1, 1, 1)), N, 1)[0, 0]
    d = np.arange(K) - K // 2
    ky, kx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    Kh = np.zeros((N, N), dtype=complex)
    for iy in range(K):
        for ix in range(K):
            Kh += t[iy, ix] * np.exp(2j * np.pi * (ky * d[iy] + kx * d[ix]) / N)
    np.testing.assert_allclose(I_k, np.abs(Kh) ** 2 * I_d, rtol=1e-10, atol=1e-8)


def test_parseval_and_dc_pixel():
    """Non-overlapping footprints: sum_k I = N^2 sum_t sum_a |y_a|^2 sum_d |t_a[d]|^2,
    and I(0) = sum_t |sum_a y_a sum_d t_a[d]|^2."""
    rng = np.random.default_rng(4)
    N, A, T, K = 32, 12, 6, 3
    pos = _integer_layout(rng, A, N, K)
    taps = rng.normal(size=(A, 1, K, K)) + 1j * rng.normal(size=(A, 1, K, K))
    xr = rng.integers(-7, 8, size=(T, 1, A, 1)); xi = rng.integers(-7, 8, size=(T, 1, A, 1))
    codes = synth.pack_4bit(xr, xi)
    gains = synth.gains_random(rng, 1, A, 1)
    I = oracle.moff_image(codes, gains, pos, taps, N, 1)[0, 0]
    y = (xr + 1j * xi)[:, 0, :, 0] * gains[0, :, 0]
    tp = np.sum(np.abs(taps[:, 0]) ** 2, axis=(1, 2))
    assert abs(I.sum() - N * N * np.sum(np.abs(y) ** 2 * tp)) < 1e-9 * I.sum()
    ts = taps[:, 0].sum(axis=(1, 2))
    assert abs(I[0, 0] - np.sum(np.abs(y @ ts) ** 2)) < 1e-9 * I[0, 0]


def test_single_antenna_delta_kernel_is_flat():
    rng = np.random.default_rng(5)
    T = 7
    xr = rng.integers(-7, 8, size=(T, 1, 1, 1)); xi = rng.integers(-7, 8, size=(T, 1, 1, 1))
    g = np.array([[[0.9 * np.exp(0.3j)]]])
    I = oracle.moff_image(synth.pack_4bit(xr, xi), g, np.array([[5.2, 9.7]]), np.ones((1, 1, 1, 1)), 16, 1)[0, 0]
    want = np.sum(np.abs((xr + 1j * xi) * g[0]) ** 2)
    np.testing.assert_allclose(I, np.full((16, 16), want), rtol=1e-13)


# ------------------------------------------------------------------ FX identity (Eqs. m1-m6)

def _small_case(seed, A, N, K, P, jones, T=6, C=2):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, N, size=(A, 2))
    if jones:
        taps = rng.normal(size=(A, 2, 2, K, K)) + 1j * rng.normal(size=(A, 2, 2, K, K))
    else:
        taps = rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K))
    codes = synth.pack_4bit(rng.integers(-8, 8, size=(T, C, A, P)), rng.integers(-8, 8, size=(T, C, A, P)))
    gains = synth.gains_random(rng, C, A, P)
    return pos, taps, codes, gains


def test_fx_identity_tiny_workload():
    """The 64-antenna tiny workload: MOFF image == FX image (visibilities of all
    2016 pairs plus autos, gridded with cross-correlated kernels) to 1e-12."""
    cfg = synth.config_tiny(n_time=64, n_chan=3)
    I = oracle.moff_image(cfg["codes"], cfg["gains"], cfg["pos"], cfg["taps"], 32, 1)
    for c in range(3):
        F = oracle.fx_image(cfg["codes"], cfg["gains"], cfg["pos"], cfg["taps"], 32, 1, channel=c)
        assert np.abs(F - I[c]).max() <= 1e-12 * np.abs(I[c]).max()


@pytest.mark.parametrize("jones", [False, True])
def test_fx_identity_dual_pol(jones):
    pos, taps, codes, gains = _small_case(6, A=10, N=16, K=3, P=2, jones=jones)
    I = oracle.moff_image(codes, gains, pos, taps, 16, 2, jones=jones)
    for c in range(2):
        F = oracle.fx_image(codes, gains, pos, taps, 16, 2, jones=jones, channel=c)
        scale = max(np.abs(I[c, 0]).max(), np.abs(I[c, 1]).max())
        assert np.abs(F - I[c]).max() <= 1e-12 * scale


def test_fx_identity_with_wrapping_footprints():
    pos, taps, codes, gains = _small_case(7, A=6, N=8, K=5, P=1, jones=False)
    pos[:3] = [[0.2, 7.6], [7.9, 0.1], [3.5, 7.5]]
    I = oracle.moff_image(codes, gains, pos, taps, 8, 1)
    F = oracle.fx_image(codes, gains, pos, taps, 8, 1, channel=1)
    assert np.abs(F - I[1]).max() <= 1e-12 * np.abs(I[1]).max()


# ------------------------------------------------------------------ invariants

def test_integer_shift_invariance_and_gain_scaling():
    pos, taps, codes, gains = _small_case(8, A=12, N=16, K=3, P=2, jones=False)
    I = oracle.moff_image(codes, gains, pos, taps, 16, 2)
    I_s = oracle.moff_image(codes, gains, pos + np.array([3.0, -5.0]), taps, 16, 2)
    np.testing.assert_allclose(I_s[:, :2], I[:, :2], rtol=1e-11, atol=1e-9)
    # cross product magnitude is also shift-invariant
    np.testing.assert_allclose(np.hypot(I_s[:, 2], I_s[:, 3]), np.hypot(I[:, 2], I[:, 3]), rtol=1e-9, atol=1e-8)
    alpha = 1.7 * np.exp(0.4j)
    I_g = oracle.moff_image(codes, gains * alpha, pos, taps, 16, 2)
    np.testing.assert_allclose(I_g, abs(alpha) ** 2 * I, rtol=1e-11, atol=1e-8)
    I_0 = oracle.moff_image(np.zeros_like(codes), gains, pos, taps, 16, 2)
    assert np.all(I_0 == 0)


def test_cross_pol_cauchy_schwarz_and_positivity():
    pos, taps, codes, gains = _small_case(9, A=12, N=16, K=3, P=2, jones=True)
    I = oracle.moff_image(codes, gains, pos, taps, 16, 2, jones=True)
    assert (I[:, 0] >= 0).all() and (I[:, 1] >= 0).all()
    assert (I[:, 2] ** 2 + I[:, 3] ** 2 <= I[:, 0] * I[:, 1] * (1 + 1e-12) + 1e-9).all()


def test_xy_is_ex_times_conj_ey():
    """Pol Y carries i times pol X (exact in 4 bits), same kernels, unit gains:
    E_y = i E_x, so XY = sum E_x conj(E_y) = -i XX (Re XY = 0, Im XY = -XX)."""
    rng = np.random.default_rng(10)
    A, N, T = 8, 16, 5
    pos = rng.uniform(0, N, size=(A, 2))
    t = rng.normal(size=(A, 1, 3, 3)) + 1j * rng.normal(size=(A, 1, 3, 3))
    taps = np.concatenate([t, t], axis=1)
    xr = rng.integers(-7, 8, size=(T, 1, A)); xi = rng.integers(-7, 8, size=(T, 1, A))
    codes = np.stack([synth.pack_4bit(xr, xi), synth.pack_4bit(-xi, xr)], axis=-1)
    I = oracle.moff_image(codes, np.ones((1, A, 2)), pos, taps, N, 2)[0]
    np.testing.assert_allclose(I[1], I[0], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(I[2], 0 * I[0], atol=1e-9 * I[0].max())
    np.testing.assert_allclose(I[3], -I[0], rtol=1e-12, atol=1e-9 * I[0].max())


def test_jones_index_order_out_then_in():
    """taps[a][p_out][p_in]: a kernel only at [p_out=0][p_in=1] puts pol-Y voltages
    into the X image and leaves Y empty."""
    rng = np.random.default_rng(11)
    A, N, T, K = 8, 16, 4, 3
    pos = rng.uniform(0, N, size=(A, 2))
    t = rng.normal(size=(A, K, K)) + 1j * rng.normal(size=(A, K, K))
    J = np.zeros((A, 2, 2, K, K), dtype=complex)
    J[:, 0, 1] = t
    codes = synth.pack_4bit(rng.integers(-7, 8, size=(T, 1, A, 2)), rng.integers(-7, 8, size=(T, 1, A, 2)))
    gains = synth.gains_random(rng, 1, A, 2)
    I = oracle.moff_image(codes, gains, pos, J, N, 2, jones=True)[0]
    I_y = oracle.moff_image(codes[..., 1:], gains[..., 1:], pos, t[:, None], N, 1)[0, 0]
    np.testing.assert_allclose(I[0], I_y, rtol=1e-11, atol=1e-9)
    assert np.abs(I[1]).max() == 0 and np.abs(I[2]).max() == 0


# ------------------------------------------------------------------ F-stage

def test_pfb_hand_summed_fixture():
    rows = read_golden("pfb_2tap_m4.txt")
    adc = np.arange(1, 9, dtype=float)[None]
    hs = {1: np.ones(8), 2: np.array([1, 0, 0, 0, 0, 0, 0, 2.0])}
    for r in rows:
        case, k, re, im = int(r[0]), int(r[1]), float(r[2]), float(r[3])
        X = oracle.pfb_spectra(adc, hs[case], 2, 4)
        assert X.shape == (1, 1, 2)
        assert abs(X[0, 0, k] - (re + 1j * im)) < 1e-12


def test_pfb_one_tap_rectangular_is_plain_fft():
    rng = np.random.default_rng(12)
    M = 64
    adc = rng.integers(-127, 128, size=(3, 2, 10 * M)).astype(float)
    X = oracle.pfb_spectra(adc, np.ones(M), 1, M)
    want = np.fft.fft(adc.reshape(3, 2, 10, M), axis=-1)[..., : M // 2]
    np.testing.assert_allclose(X, want, rtol=0, atol=1e-9)


def test_pfb_window_hand_values():
    """The window's coefficients for 2 taps of M = 4, against the closed forms
    worked by hand in tests/golden/pfb_window_2tap_m4.txt: both Hann endpoints
    vanish (L - 1 in the cosine's denominator, not L) and the sinc is centred
    at (L - 1) / 2 (half a sample off would break the symmetry and move every
    value)."""
    rows = read_golden("pfb_window_2tap_m4.txt")
    want = np.array([float(r[1]) for r in rows])
    assert [int(r[0]) for r in rows] == list(range(8))
    h = oracle.pfb_window(2, 4)
    assert h.shape == (8,)
    np.testing.assert_allclose(h, want, rtol=1e-13, atol=1e-15)


def test_pfb_window_channel_response():
    """Windowed-sinc PFB: a tone at a channel centre keeps >= 99 % of its power in
    that channel; at a channel edge the two neighbours see it about equally."""
    M, P = 256, 8
    h = oracle.pfb_window(P, M)
    assert np.allclose(h, h[::-1])
    n = np.arange((P + 20) * M)
    k0 = 37
    X = oracle.pfb_spectra(np.cos(2 * np.pi * k0 * n / M)[None], h, P, M)[0]
    pw = np.sum(np.abs(X) ** 2, axis=0)
    assert pw[k0] >= 0.99 * pw.sum()
    X = oracle.pfb_spectra(np.cos(2 * np.pi * (k0 + 0.5) * n / M)[None], h, P, M)[0]
    pw = np.sum(np.abs(X) ** 2, axis=0)
    assert abs(pw[k0] / pw[k0 + 1] - 1) < 0.05
    assert (pw[k0] + pw[k0 + 1]) >= 0.98 * pw.sum()


def test_channelise_layout_and_codes():
    rng = np.random.default_rng(13)
    M, P = 32, 4
    adc = synth.adc_stream(rng, 3, 2, (P + 5) * M)
    h = oracle.pfb_window(P, M)
    codes, X = oracle.channelise(adc, h, P, M, 0.05)
    assert codes.shape == (6, M // 2, 3, 2) and X.shape == codes.shape
    z = oracle.unpack_4bit(codes)
    re, im = oracle.quantise_4bit(X, 0.05)
    np.testing.assert_array_equal(z.real, re)
    np.testing.assert_array_equal(z.imag, im)
    # a frame is built from its own and the next P-1 blocks of M samples
    Xa = oracle.pfb_spectra(adc[1, 0, 2 * M:(2 + P) * M], h, P, M)[0]
    np.testing.assert_allclose(X[2, :, 1, 0], Xa, atol=1e-9)


# ------------------------------------------------------------------ metric

def test_max_norm_err_denominators():
    ref = np.zeros((1, 4, 2, 2)); ref[0, 0] = 4.0; ref[0, 1] = 2.0; ref[0, 2] = 1.0; ref[0, 3] = 1.0
    img = ref.copy(); img[0, 2, 0, 0] += 0.4; img[0, 1, 1, 1] += 0.2
    e = oracle.max_norm_err(img, ref)[0]
    np.testing.assert_allclose(e, [0.0, 0.1, 0.1, 0.0])


# ------------------------------------------------------------------ absolute placement, per-pol kernels

def test_grid_placement_hand_example():
    """Antenna at (x, y) = (5.2, 9.7) -> anchor (5, 10); a 3x3 kernel t[dy][dx]
    lands on rows 9..11 and columns 4..6 with G[9 + dy][4 + dx] = t[dy][dx].
    Antenna at (0.3, 15.6) -> anchor (0, 16) wraps on N = 16 to rows 15, 0, 1
    and columns 15, 0, 1 (worked by hand)."""
    t = (np.arange(9).reshape(3, 3) + 1) * (1 + 0.5j)
    for pos, rows, cols in [((5.2, 9.7), [9, 10, 11], [4, 5, 6]),
                            ((0.3, 15.6), [15, 0, 1], [15, 0, 1])]:
        W = oracle.grid_matrix(np.array([pos]), t[None, None], 16, 1)
        G = oracle.grid(np.ones((1, 1, 1)), W, 16, 1)[0, 0]
        want = np.zeros((16, 16), dtype=complex)
        for dy in range(3):
            for dx in range(3):
                want[rows[dy], cols[dx]] = t[dy, dx]
        np.testing.assert_array_equal(G, want)


def test_dual_pol_products_are_per_pol_images():
    """Without Jones coupling, XX and YY are the single-pol images of each pol
    through that pol's own kernel."""
    pos, taps, codes, gains = _small_case(14, A=10, N=16, K=3, P=2, jones=False)
    I = oracle.moff_image(codes, gains, pos, taps, 16, 2)
    for p in range(2):
        Ip = oracle.moff_image(codes[..., p:p + 1], gains[..., p:p + 1], pos, taps[:, p:p + 1], 16, 1)
        np.testing.assert_allclose(I[:, p], Ip[:, 0], rtol=1e-12, atol=1e-9)


# ----------------------------------------------------------------------------- feedback calibration (Sec. 6)

def _fb_case(seed, A=24, N=32, K=3, P=2, T=9):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(3, N - 3, size=(A, 2))
    taps = rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K))
    y = rng.normal(size=(T, A, P)) + 1j * rng.normal(size=(T, A, P))
    return pos, taps, y


def test_feedback_antenna_shares_sum_to_the_image_pixel():
    """FBeq1 = sum over antennas of FBeq2: the image pixel (grid + transform)
    must equal the sum of the antennas' beam-weighted voltages."""
    pos, taps, y = _fb_case(1)
    for k in [(0, 0), (5, 11), (31, 2)]:
        R, S = oracle.feedback_sums_y(y, pos, taps, 32, k)
        assert np.allclose(R.sum(axis=0), S, rtol=1e-12, atol=0)
        assert np.abs(R.sum(axis=0).imag).max() <= 1e-10 * S.max()


def test_feedback_fbeq3_by_antenna_pairs():
    """FBeq3: <|E|^2> - <E conj(c_i)> = sum over pairs (j, k != i) of <c_j conj(c_k)>,
    with c the per-antenna pixel shares taken from single-antenna images."""
    pos, taps, y = _fb_case(2, A=7, N=16, K=3, P=1, T=5)
    k = (3, 9)
    R, S = oracle.feedback_sums_y(y, pos, taps, 16, k)
    # per-antenna shares from the imaging path run on one antenna at a time
    c = np.zeros((y.shape[0], 7), dtype=complex)
    for a in range(7):
        ya = np.zeros_like(y)
        ya[:, a] = y[:, a]
        W = oracle.grid_matrix(pos, taps, 16, 1)
        c[:, a] = oracle.sky_transform(oracle.grid(ya, W, 16, 1))[:, 0, k[1], k[0]]
    for i in range(7):
        pairs = sum(np.sum(c[:, j] * np.conj(c[:, kk])) for j in range(7) for kk in range(7) if kk != i)
        assert abs((S[0] - R[i, 0]) - pairs) <= 1e-10 * S[0]


def test_feedback_point_source_closed_form():
    """Delta kernels, integer anchors, unit gains, one source at theta_s with
    phases exp(-2 pi i p.theta_s/N) that are multiples of pi/2 (exact 4-bit):
    E(theta_s) = A x, so N conj(R)/S = 1 and the gain error estimate is 0;
    the printed factor 2N would give -g instead."""
    N, A, T = 32, 12, 4
    rng = np.random.default_rng(3)
    cells = rng.choice(N * N, size=A, replace=False)
    pos = np.stack([cells % N, cells // N], axis=1).astype(float)
    th = (8, 0)                                   # theta_s: phases i^(-px)
    x = 7 * np.exp(-2j * np.pi * (pos[:, 0] * th[0] + pos[:, 1] * th[1]) / N)
    re, im = np.rint(x.real).astype(int), np.rint(x.imag).astype(int)
    codes = np.repeat(synth.pack_4bit(re, im)[None, None, :, None], T, axis=0)   # [T, 1, A, 1]
    gains = np.ones((1, A, 1), complex)
    taps = np.ones((A, 1, 1, 1), complex)
    R, S = oracle.feedback_sums(codes, gains, pos, taps, N, th)
    assert np.isclose(S[0, 0], T * 49 * A ** 2)          # E(theta_s) = 7 A per sample
    assert np.allclose(R[0, :, 0], T * 49 * A)           # E conj(x_a B_a) = 7 A * 7
    assert np.allclose(oracle.feedback_delta(R, S, gains, A), 0, atol=1e-12)
    assert np.allclose(gains * (1 - 2 * A * np.conj(R) / S[:, None, :]), -gains)


def _simulated_step(eps, factor, conj=True, seed=4):
    """One feedback step on a simulated point source with residual gain errors
    (1 + eps); returns the largest relative residual before and after."""
    N, A, T = 32, len(eps), 64
    rng = np.random.default_rng(seed)
    cells = rng.choice(N * N, size=A, replace=False)
    pos = np.stack([cells % N, cells // N], axis=1).astype(float)
    th = (5, 13)
    geo = np.exp(-2j * np.pi * (pos[:, 0] * th[0] + pos[:, 1] * th[1]) / N)
    h = (0.8 + 0.4 * rng.random(A)) * np.exp(2j * np.pi * rng.random(A))   # instrument gains
    s = rng.normal(size=T) + 1j * rng.normal(size=T)                        # source signal
    x = (s[:, None] * (h * geo)[None, :])[:, :, None]                       # [T, A, 1]
    g = (1 / h) * (1 + np.asarray(eps))
    taps = np.ones((A, 1, 1, 1), complex)
    R, S = oracle.feedback_sums_y(x * g[None, :, None], pos, taps, N, th)
    ratio = np.conj(R[:, 0]) if conj else R[:, 0]
    g_new = g + g * (1 - factor * ratio / S[0])
    spread = lambda a: np.abs(a / a.mean() - 1).max()
    return spread(g * h), spread(g_new * h)


def test_feedback_update_removes_a_simulated_gain_error():
    """The N reading with the conjugated ratio cancels a 5 % amplitude and phase
    error to second order in one step; the printed 2N and the unconjugated
    ratio do not converge."""
    rng = np.random.default_rng(5)
    eps = 0.05 * (rng.normal(size=20) + 1j * rng.normal(size=20)) / np.sqrt(2)
    before, after = _simulated_step(eps, factor=20)
    assert before > 0.05 and after < 0.15 * before
    b2, a2 = _simulated_step(eps, factor=40)
    assert a2 > 0.9 * b2
    b3, a3 = _simulated_step(1j * np.abs(eps), factor=20, conj=False)
    assert a3 > 0.9 * b3


# ----------------------------------------------------------------------------- autocorrelation subtraction

@pytest.mark.parametrize("P,K", [(1, 3), (2, 3)])
def test_baselines_only_image_is_image_minus_autos(P, K):
    """The FX route without the a = b visibilities equals the MOFF image minus
    the sum of single-antenna images (two independent routes)."""
    rng = np.random.default_rng(20 + P)
    A, N, T = 9, 16, 6
    pos = rng.uniform(2, 14, size=(A, 2))
    taps = rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K))
    codes = synth.pack_4bit(rng.integers(-7, 8, size=(T, 1, A, P)), rng.integers(-7, 8, size=(T, 1, A, P)))
    gains = synth.gains_random(rng, 1, A, P)
    full = oracle.moff_image(codes, gains, pos, taps, N, P)[0]
    autos = oracle.auto_image(codes, gains, pos, taps, N, P)
    cross = oracle.fx_image(codes, gains, pos, taps, N, P, autos=False)
    assert np.allclose(full - autos, cross, rtol=0, atol=1e-9 * np.abs(full).max())
    # the autocorrelation image does not depend on where the antennas are
    moved = oracle.auto_image(codes, gains, pos + rng.integers(-2, 3, size=(A, 2)), taps, N, P)
    assert np.allclose(moved, autos, rtol=0, atol=1e-9 * np.abs(autos).max())


def test_autos_of_a_delta_antenna_are_flat():
    """One antenna, delta kernel: its image is flat at sum_t |y|^2 (and so its
    baselines-only image is zero)."""
    rng = np.random.default_rng(30)
    codes = synth.pack_4bit(rng.integers(-7, 8, size=(5, 1, 1, 1)), rng.integers(-7, 8, size=(5, 1, 1, 1)))
    gains = np.array([[[1.5 - 0.5j]]])
    y = oracle.calibrate(oracle.unpack_4bit(codes[:, 0]), gains[0])
    autos = oracle.auto_image(codes, gains, np.array([[3.0, 4.0]]), np.ones((1, 1, 1, 1)), 8, 1)
    assert np.allclose(autos, np.sum(np.abs(y) ** 2))
    cross = oracle.fx_image(codes, gains, np.array([[3.0, 4.0]]), np.ones((1, 1, 1, 1)), 8, 1, autos=False)
    assert np.abs(cross).max() == 0.0
