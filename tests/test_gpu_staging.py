"""Host voltage blocks staged by channel segments (moff_submit with a host
pointer): the imaging of each channel chunk waits only for its own segment's
copy.  The launches are those of a device-input submit, so the image must be
bit-identical to it, on the FP32 path and on the tensor-core gridding route.
The second block is below the segmenting threshold and is copied whole."""
import numpy as np
import pytest

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


def run(pos, taps, N, C, P, gains, blocks, host, fp16tc=False):
    with moff.Plan(pos, taps, N, C, P, fp16tc=fp16tc) as pl:
        info = pl.info()
        assert pl.route() == ("fp16_tcgrid" if fp16tc else "fp32")
        pl.set_gains(gains)
        for b in blocks:
            pl.submit(b.cpu().numpy() if host else b)
        img, n = pl.read_image()
    return img, n, info


@pytest.mark.parametrize("fp16tc", [False, True])
def test_host_block_by_channel_segments_equals_device_input(monkeypatch, fp16tc):
    rng = np.random.default_rng(501)
    side, N, K, P, C = 48, 256, 7, 2, 48
    pos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N / 2 - side, N / 2 - side))
    A = pos.shape[0]
    taps = synth.taps_gaussian(rng, pos, K, 1.2, n_pol=P).astype(np.complex64)
    gains = synth.gains_random(rng, C, A, P).astype(np.complex64)
    # blocks of 22 MB and 4.4 MB, several channel chunks each
    blocks = [synth.device_codes(502, 100, C, A, P), synth.device_codes(503, 20, C, A, P)]
    # (the second block still spans channel chunks: below 8 MB it is copied whole)
    monkeypatch.setenv("MOFF_SCRATCH_MB", "300" if fp16tc else "24")
    dev, nd, info = run(pos, taps, N, C, P, gains, blocks, host=False, fp16tc=fp16tc)
    assert info["chan_chunk"] < C, info
    host, nh, _ = run(pos, taps, N, C, P, gains, blocks, host=True, fp16tc=fp16tc)
    assert nd == nh == 120
    assert np.array_equal(dev, host)
