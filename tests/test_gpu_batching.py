"""Batching: whole blocks replayed as CUDA graphs (MOFF_GRAPH) and the
gridding shape picked by the autotuner (MOFF_AUTOTUNE).

A graph replays exactly the launches a direct submit makes, so images must be
bit-identical with and without graphs; the autotuner only changes the
gridding kernel's shape, so its images are held to the FP32 bar (1e-5)
against the FP64 oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def array(seed, A, N, K, P, C):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, N * 0.7, size=(A, 2)) + N * 0.15
    taps = c64(rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K)))
    gains = c64(synth.gains_random(rng, C, A, P))
    return pos, taps, gains


def codes(seed, T, C, A, P):
    rng = np.random.default_rng(seed)
    re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -7, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -7, 7).astype(int)
    return synth.pack_4bit(re, im)


def run(pos, taps, gains, N, C, P, blocks, **kw):
    with moff.Plan(pos, taps, N, C, P, **kw) as pl:
        pl.set_gains(gains)
        for b in blocks:
            pl.submit(b)
        img, n = pl.read_image()
    return img, n


@pytest.mark.parametrize("N,P,K,A", [(64, 2, 5, 200), (128, 1, 7, 300)])
def test_graph_replay_is_bit_identical(N, P, K, A):
    C = 5
    pos, taps, gains = array(40 + N, A, N, K, P, C)
    host = [codes(41, 37, C, A, P), codes(42, 37, C, A, P), codes(43, 12, C, A, P)]
    dev = torch.from_numpy(codes(44, 37, C, A, P)).cuda()
    torch.cuda.synchronize()
    # device block submitted three times (capture, then two replays), host blocks
    # through both staging buffers, and a second block length
    blocks = [dev, host[0], dev, host[1], host[2], dev, host[0]]
    a, na = run(pos, taps, gains, N, C, P, blocks)
    b, nb = run(pos, taps, gains, N, C, P, blocks, graph=True)
    assert na == nb
    assert np.array_equal(a, b)


def test_graph_replay_of_the_fstage_path_and_filter_change():
    A, P, C, N, ntaps = 6, 2, 64, 32, 4
    rng = np.random.default_rng(50)
    pos = rng.uniform(4, 28, size=(A, 2))
    taps = c64(rng.normal(size=(A, P, 3, 3)) + 1j * rng.normal(size=(A, P, 3, 3)))
    adc = torch.from_numpy(synth.adc_stream(rng, A, P, (ntaps + 9) * 2 * C, sigma=20.0)).cuda()
    torch.cuda.synchronize()
    out = []
    for graph in (False, True):
        with moff.Plan(pos, taps, N, C, P, fstage=True, graph=graph) as pl:
            pl.set_fstage(ntaps, None, 0.02)
            pl.submit_adc(adc)
            pl.submit_adc(adc)
            pl.set_fstage(ntaps, None, 0.05)      # captured launches must not keep the old scale
            pl.submit_adc(adc)
            out.append(pl.read_image())
    assert out[0][1] == out[1][1] == 30
    assert np.array_equal(out[0][0], out[1][0])


def test_timing_on_bypasses_graphs_and_agrees():
    pos, taps, gains = array(60, 120, 64, 5, 2, 3)
    blk = torch.from_numpy(codes(61, 20, 3, 120, 2)).cuda()
    torch.cuda.synchronize()
    with moff.Plan(pos, taps, 64, 3, 2, graph=True) as pl:
        pl.set_gains(gains)
        pl.submit(blk)                      # captured and replayed
        pl.set_timing(True)
        pl.submit(blk)                      # direct launches, timed
        ms, n = pl.timing(1)
        assert n >= 1 and ms > 0.0
        pl.set_timing(False)
        pl.submit(blk)                      # replay again
        img, ns = pl.read_image()
    ref, nr = run(pos, taps, gains, 64, 3, 2, [blk, blk, blk])
    assert ns == nr == 60
    assert np.array_equal(img, ref)


def test_autotuned_plan_matches_oracle_and_is_cached():
    A, N, K, P, C, T = 400, 128, 7, 2, 3, 25
    pos, taps, gains = array(70, A, N, K, P, C)
    blk = codes(71, T, C, A, P)
    with moff.Plan(pos, taps, N, C, P, autotune=True) as pl:
        tu = pl.tuning()
        assert tu["source"] in (1, 2) and tu["time_batch"] in (1, 2, 4, 8) and tu["staged"] in (0, 1)
        assert tu["cells_per_lane"] in (1, 2, 4) and tu["wide_rows"] in (0, 1)
        pl.set_gains(gains)
        pl.submit(blk)
        img, n = pl.read_image()
    ref = oracle.moff_image(blk, gains, pos, taps, N, P)
    err = oracle.max_norm_err(img, ref)
    print("autotuned shape", tu, "max-normalised error", float(err.max()))
    assert err.max() <= TOL32
    with moff.Plan(pos, taps, N, C, P, autotune=True) as pl2:
        tu2 = pl2.tuning()
    assert tu2["source"] == 2 and (tu2["time_batch"], tu2["staged"], tu2["cells_per_lane"], tu2["wide_rows"]) == (
        tu["time_batch"], tu["staged"], tu["cells_per_lane"], tu["wide_rows"])
    with moff.Plan(pos, taps, N, C, P) as pl3:
        assert pl3.tuning()["source"] == 0


def test_tuning_cache_file_is_shared_between_processes(tmp_path):
    path = str(tmp_path / "tune.txt")
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np, paper_0812_3669_gb300 as moff\n"
        "rng = np.random.default_rng(80)\n"
        "pos = rng.uniform(10, 50, size=(150, 2)); taps = np.ones((150, 1, 5, 5), complex)\n"
        "pl = moff.Plan(pos, taps, 64, 2, 1, autotune=True)\n"
        "t = pl.tuning(); print('SRC', t['source'], t['time_batch'], t['staged'], t['cells_per_lane'], t['wide_rows'])\n" % ROOT)
    env = dict(os.environ, MOFF_TUNE_CACHE=path)
    outs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append([ln for ln in r.stdout.splitlines() if ln.startswith("SRC")][0].split())
    assert outs[0][1] == "1" and outs[1][1] == "2"
    assert outs[0][2:] == outs[1][2:]
    assert open(path).read().count("\n") == 1
