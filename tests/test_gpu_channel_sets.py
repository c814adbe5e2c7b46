"""Channel-dependent antenna positions and kernels (moff_set_channel_groups) vs
the FP64 oracle.

Positions in wavelengths scale with frequency, so each channel may see its
own set of positions and kernels.  Every channel must match the oracle run
with its set at the FP32 bar (1e-5 max-normalised), and a channel must come out
bit-identical to a plan created with its set when both grid with one shape.
Calibrator sums, autocorrelation subtraction and graph replays follow the sets.
"""
import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def scaled_sets(seed, A, N, K, P, scales, jones=False):
    """One reference layout in the middle of the grid, scaled about the grid centre
    per set (frequency / reference frequency), with each set's own kernels."""
    rng = np.random.default_rng(seed)
    base = rng.uniform(-0.3 * N, 0.3 * N, size=(A, 2))
    pos = np.stack([N / 2 + base * s for s in scales])
    shape = (A, 2, 2, K, K) if jones else (A, P, K, K)
    taps = c64(rng.normal(size=(len(scales),) + shape) + 1j * rng.normal(size=(len(scales),) + shape))
    return pos, taps


def codes_for(seed, T, C, A, P):
    rng = np.random.default_rng(seed)
    re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -8, 7).astype(int)
    return synth.pack_4bit(re, im), c64(synth.gains_random(rng, C, A, P))


@pytest.mark.parametrize("N,P,K,A,jones", [(64, 2, 5, 120, False), (128, 1, 7, 200, False),
                                          (64, 2, 3, 40, True), (32, 1, 3, 50, False)])
def test_channel_sets_match_the_oracle(N, P, K, A, jones):
    C, T = 5, 37
    grp = [0, 1, 2, 1, 0]
    pos, taps = scaled_sets(800 + N + K, A, N, K, P, [1.0, 1.2, 0.85], jones)
    codes, gains = codes_for(801 + N, T, C, A, P)
    with moff.Plan(pos[0], taps[0], N, C, P, jones=jones) as pl:
        pl.set_gains(gains)
        pl.set_channel_groups(pos, taps, grp)
        pl.submit(codes[:20])
        pl.submit(codes[20:])
        img, n = pl.read_image()
    assert n == T
    ref = oracle.moff_image_sets(codes, gains, pos, taps, grp, N, P, jones=jones)
    err = oracle.max_norm_err(img, ref)
    print(f"N={N} P={P} jones={jones}: max-normalised error {err.max():.2e}")
    assert err.max() <= TOL32
    # the sets really differ: channel 1 is not the image of set 0
    alt = oracle.moff_image(codes, gains, pos[0], taps[0], N, P, jones=jones, channels=[1])
    assert oracle.max_norm_err(img[1:2], alt).max() > 1e-2


@pytest.mark.parametrize("quads", ["0", "1"])
def test_a_channel_equals_a_plan_created_with_its_set(monkeypatch, quads):
    """Same gridding shape (forced by the environment rule knobs; pair lanes or
    2 x 2 block lanes): the channels of set 1 in a two-set plan are bit-identical
    to a plan created with set 1."""
    N, P, K, A, C, T = 64, 2, 5, 150, 4, 29
    monkeypatch.setenv("MOFF_GRID_PAIRS", "1")
    monkeypatch.setenv("MOFF_GRID_QUADS", quads)
    monkeypatch.setenv("MOFF_GRID_STAGE", "0")
    pos, taps = scaled_sets(830, A, N, K, P, [1.0, 1.1])
    codes, gains = codes_for(831, T, C, A, P)
    grp = [0, 1, 1, 0]
    with moff.Plan(pos[0], taps[0], N, C, P) as pl:
        pl.set_gains(gains)
        pl.set_channel_groups(pos, taps, grp)
        tu = pl.tuning()
        pl.submit(codes)
        two, _ = pl.read_image()
    with moff.Plan(pos[1], taps[1], N, C, P) as p1:
        t1 = p1.tuning()
        p1.set_gains(gains)
        p1.submit(codes)
        one, _ = p1.read_image()
    assert (tu["time_batch"], tu["cells_per_lane"], tu["staged"]) == (t1["time_batch"], t1["cells_per_lane"], t1["staged"])
    assert tu["cells_per_lane"] == (4 if quads == "1" else 2)
    assert np.array_equal(two[1:3], one[1:3])


def test_replace_switch_back_and_graph_replay():
    """One set replacing the creation-time set, then back; graph replays of the same
    block before and after each change equal direct launches."""
    N, P, K, A, C, T = 64, 2, 5, 100, 3, 24
    pos, taps = scaled_sets(840, A, N, K, P, [1.0, 1.3])
    codes, gains = codes_for(841, T, C, A, P)
    dev = torch.from_numpy(codes).cuda()
    torch.cuda.synchronize()
    out = []
    for graph in (False, True):
        with moff.Plan(pos[0], taps[0], N, C, P, graph=graph) as pl:
            pl.set_gains(gains)
            pl.submit(dev)
            a, _ = pl.read_image(reset=True)
            pl.set_channel_groups(pos[1:], taps[1:])            # one set for every channel
            pl.submit(dev)
            b, _ = pl.read_image(reset=True)
            pl.set_channel_groups(pos[:1], taps[:1], [0] * C)    # back to the creation-time set
            pl.submit(dev)
            c, _ = pl.read_image(reset=True)
        out.append((a, b, c))
    assert all(np.array_equal(x, y) for x, y in zip(out[0], out[1]))
    a, b, c = out[0]
    assert np.array_equal(a, c)
    assert oracle.max_norm_err(a, oracle.moff_image(codes, gains, pos[0], taps[0], N, P)).max() <= TOL32
    assert oracle.max_norm_err(b, oracle.moff_image(codes, gains, pos[1], taps[1], N, P)).max() <= TOL32


def test_feedback_and_autocorr_follow_the_sets():
    N, P, K, A, C, T = 64, 2, 5, 90, 3, 40
    grp = [1, 0, 1]
    pos, taps = scaled_sets(850, A, N, K, P, [1.0, 1.25])
    codes, gains = codes_for(851, T, C, A, P)
    k = (9, 50)
    with moff.Plan(pos[0], taps[0], N, C, P) as pl:
        pl.set_gains(gains)
        pl.set_calibrator(*k)
        pl.set_autocorr(True)
        pl.set_channel_groups(pos, taps, grp)
        pl.submit(codes)
        R, S, n = pl.read_feedback()
        cross, nc = pl.read_image_cross()
    assert n == nc == T
    full = oracle.moff_image_sets(codes, gains, pos, taps, grp, N, P)
    for c, g in enumerate(grp):
        Ro, So = oracle.feedback_sums(codes, gains, pos[g], taps[g], N, k, channels=[c])
        assert (np.abs(S[c] - So[0]) / So[0]).max() <= TOL32
        assert (np.abs(R[c] - Ro[0]).max(axis=0) / np.abs(Ro[0]).max(axis=0)).max() <= TOL32
        auto = oracle.auto_image(codes, gains, pos[g], taps[g], N, P, channel=c)
        den = np.abs(full[c]).reshape(-1, N * N).max(axis=-1)
        err = np.abs(cross[c] - (full[c] - auto)).reshape(-1, N * N).max(axis=-1) / den
        assert err.max() <= TOL32


def test_errors_leave_the_plan_unchanged():
    N, P, K, A, C, T = 32, 1, 3, 30, 2, 10
    pos, taps = scaled_sets(860, A, N, K, P, [1.0, 1.1])
    codes, gains = codes_for(861, T, C, A, P)
    with moff.Plan(pos[0], taps[0], N, C, P) as pl:
        pl.set_gains(gains)
        for args, status in [((pos, taps, [0, 2]), -1),            # set index out of range
                             ((pos, taps, None), -1),              # two sets, no map
                             ((np.concatenate([pos] * 2), np.concatenate([taps] * 2), [0, 1]), -1)]:   # G > C
            with pytest.raises(moff.MoffError) as e:
                pl.set_channel_groups(*args)
            assert e.value.status == status
        bad = pos.copy()
        bad[1, 3, 0] = np.nan
        with pytest.raises(moff.MoffError) as e:
            pl.set_channel_groups(bad, taps, [0, 1])
        assert e.value.status == -1
        pl.submit(codes)
        img, _ = pl.read_image()
    ref = oracle.moff_image(codes, gains, pos[0], taps[0], N, P)
    assert oracle.max_norm_err(img, ref).max() <= TOL32
    rng = np.random.default_rng(862)
    tpos = rng.uniform(30, 98, size=(100, 2))
    ttaps = np.ones((100, 2, 5, 5), complex)
    with moff.Plan(tpos, ttaps, 128, 2, 2, fp16tc=True) as pt:
        with pytest.raises(moff.MoffError) as e:
            pt.set_channel_groups(tpos[None], ttaps[None])
        assert e.value.status == -1


def test_edge_padding_samples_the_same_image():
    """Image oversampling by edge padding (Sec. 4): the same array on a grid twice
    as large gives the same image at every second pixel (footprints wrap on
    neither grid)."""
    N, P, K, A, C, T = 64, 2, 5, 80, 2, 30
    rng = np.random.default_rng(870)
    pos = rng.uniform(6, N - 7, size=(A, 2))
    taps = c64(rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K)))
    codes, gains = codes_for(871, T, C, A, P)
    imgs = []
    for n in (N, 2 * N):
        with moff.Plan(pos, taps, n, C, P) as pl:
            pl.set_gains(gains)
            pl.submit(codes)
            imgs.append(pl.read_image()[0])
    small, big = imgs
    err = oracle.max_norm_err(big[:, :, ::2, ::2], small)
    assert err.max() <= 2 * TOL32
    assert oracle.max_norm_err(big, oracle.moff_image(codes, gains, pos, taps, 2 * N, P)).max() <= TOL32
