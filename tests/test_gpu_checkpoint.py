"""Checkpoint and resume of an integration (moff_export_accumulators /
moff_import_accumulators): the FP64 sums of the first blocks, exported from one
plan and imported into a fresh one that takes the remaining blocks, equal the
sums of one plan that took every block -- bit for bit, since each block adds
to the same FP64 values in the same order -- on the FP32 path and across
routes (an FP32 checkpoint continued on the FP16 route stays within that
route's tolerance of the oracle)."""
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


def case(seed, A, N, K, P, C, T_list):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, N * 0.7, size=(A, 2)) + N * 0.15
    taps = (rng.normal(size=(A, P, K, K)) + 1j * rng.normal(size=(A, P, K, K))).astype(np.complex64)
    gains = synth.gains_random(rng, C, A, P).astype(np.complex64)
    blocks = []
    for T in T_list:
        re = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -7, 7).astype(int)
        im = np.clip(np.rint(rng.normal(0, 2.5, size=(T, C, A, P))), -7, 7).astype(int)
        blocks.append(synth.pack_4bit(re, im))
    return pos, taps, gains, blocks


@pytest.mark.parametrize("device_buffers", [False, True])
def test_resume_equals_uninterrupted(device_buffers):
    N, P, C = 64, 2, 3
    pos, taps, gains, blocks = case(811, 150, N, 5, P, C, [30, 21, 17])
    with moff.Plan(pos, taps, N, C, P) as pl:
        pl.set_gains(gains)
        for b in blocks:
            pl.submit(b)
        whole, nw = pl.read_image()
    with moff.Plan(pos, taps, N, C, P) as first:
        first.set_gains(gains)
        for b in blocks[:2]:
            first.submit(b)
        buf = torch.empty((C, 4, N, N), dtype=torch.float64, device="cuda") if device_buffers else None
        acc, n = first.export_accumulators(buf)
        if device_buffers:
            torch.cuda.synchronize()
    assert n == 51
    with moff.Plan(pos, taps, N, C, P) as second:
        second.set_gains(gains)
        second.import_accumulators(acc, n)
        second.submit(blocks[2])
        resumed, nr = second.read_image()
    assert nr == nw == 68
    assert np.array_equal(resumed, whole)


def test_checkpoint_continues_on_another_route_and_rejects_bad_buffers():
    """Sums exported by an FP32 plan continue on the FP16 tensor-core route (dense lattice
    on the 256 grid): the image stays within the FP16 tolerance of the oracle."""
    rng = np.random.default_rng(812)
    side, N, K, P, C = 48, 256, 7, 2, 2
    pos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N / 2 - side, N / 2 - side))
    taps = synth.taps_gaussian(rng, pos, K, 1.2, n_pol=P).astype(np.complex64)
    gains = synth.gains_random(rng, C, pos.shape[0], P).astype(np.complex64)
    re = np.clip(np.rint(rng.normal(0, 2, size=(20, C, pos.shape[0], P))), -7, 7).astype(int)
    im = np.clip(np.rint(rng.normal(0, 2, size=(20, C, pos.shape[0], P))), -7, 7).astype(int)
    codes = synth.pack_4bit(re, im)
    with moff.Plan(pos, taps, N, C, P) as p32:
        p32.set_gains(gains)
        p32.submit(codes[:12])
        acc, n = p32.export_accumulators()
        with pytest.raises(ValueError):
            p32.export_accumulators(np.empty(10, dtype=np.float64))
        with pytest.raises(ValueError):
            p32.import_accumulators(acc.astype(np.float32), n)
    with moff.Plan(pos, taps, N, C, P, fp16tc=True) as p16:
        assert p16.route() == "fp16_tcgrid"
        p16.set_gains(gains)
        p16.import_accumulators(acc, n)
        p16.submit(codes[12:])
        img, n16 = p16.read_image()
    assert n16 == 20
    ref = oracle.moff_image(codes, gains.astype(np.complex128), pos, taps.astype(np.complex128), N, P)
    err = oracle.max_norm_err(img, ref)
    print(f"FP32 checkpoint continued on the FP16 route: max-normalised error {float(err.max()):.2e}")
    assert err.max() <= 3e-3
