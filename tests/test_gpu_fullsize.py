"""The FP16 tensor-core path on the dense workloads at full size, against the
FP64 oracle, at the reduced-precision bar (max-normalised error <= 3e-3 per
image; see test_gpu_dft.py for the error budget).

* Filled aperture (16384 antennas on a 128 x 128 lambda lattice, dual pol, 7x7
  kernels, 512 grid): 8 seeded channels over a whole 2000-sample integration,
  so 16 chunks of 128 samples fold into the FP64 accumulators.
* Wide field (32768 antennas, 9x9 Jones kernels with a w-phase, x wrapping the
  grid): 2 channels x 24 samples.
Each test prints its per-image errors.
"""
import numpy as np
import pytest

import oracle
import paper_0812_3669_gb300 as moff
import synth
from oracle_pool import moff_image_channels

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


def image(cfg, C, codes_d, gains):
    with moff.Plan(cfg["pos"], cfg["taps"], cfg["grid_n"], C, 2, jones=cfg["jones"], fp16tc=True) as pl:
        assert pl.route() == "fp16_tcgrid", pl.route()
        pl.set_gains(gains)
        pl.submit(codes_d)
        img, n = pl.read_image()
    assert n == codes_d.shape[0] and np.isfinite(img).all()
    return img


def report(img, ref, label):
    err = oracle.max_norm_err(img, ref)
    print(f"{label}: max-normalised error per image (XX YY ReXY ImXY)")
    for c in range(err.shape[0]):
        print(f"  channel {c}: " + " ".join(f"{e:.2e}" for e in err[c]))
    assert err.max() <= TOL16, err
    return err


def test_filled_aperture_full_integration_8_channels():
    cfg = synth.config_precision(n_chan=8)
    T, C, A, P, N = 2000, 8, cfg["pos"].shape[0], 2, cfg["grid_n"]
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    cfg["taps"] = taps
    codes_d = synth.device_codes(8123669 + 210, T, C, A, P)
    img = image(cfg, C, codes_d, gains)
    ref = moff_image_channels(codes_d.cpu().numpy(), gains, cfg["pos"], taps, N, P)
    report(img, ref, "filled aperture, 8 channels x 2000 samples")


def test_widefield_jones_sample():
    cfg = synth.config_widefield(n_chan=2)
    T, C, A, P, N = 24, 2, cfg["pos"].shape[0], 2, cfg["grid_n"]
    taps, gains = c64(cfg["taps"]), c64(cfg["gains"])
    cfg["taps"] = taps
    codes_d = synth.device_codes(8123669 + 211, T, C, A, P)
    img = image(cfg, C, codes_d, gains)
    ref = oracle.moff_image(codes_d.cpu().numpy(), gains, cfg["pos"], taps, N, P, jones=True)
    report(img, ref, "wide field Jones, 2 channels x 24 samples")
