"""Voltage decoding bit for bit on the GPU, and the bounded host wait.

Decoding (the 4-bit format of the voltages Eq. m6 starts from): 256 antennas
on distinct cells hold all 256 byte codes; with one-cell (delta) kernels and
unit gains the gridded field at each antenna's cell is its decoded voltage,
an exact small integer in FP32, so it must equal the two's-complement nibbles
exactly -- on the FP32 gridding (shared by the factored-DFT tensor-core
route) and in the FP16 voltage planes of the row-spectrum route (there times
the channel's power-of-two scale, still exact).

Bounded wait: moff_read_image with timeout_ms = 0 behind queued GPU work
returns MOFF_ETIMEDOUT (-5) and leaves the plan as it was.
"""
import numpy as np
import pytest

import paper_0812_3669_gb300 as moff
import synth
from conftest import read_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    moff.build()
    yield


def all_codes():
    re, im = np.meshgrid(np.arange(-8, 8), np.arange(-8, 8), indexing="ij")
    re, im = re.ravel(), im.ravel()
    return synth.pack_4bit(re, im), re, im


def lattice(n_side, spacing, offset=0.0):
    a = np.arange(n_side * n_side)
    return np.stack([offset + spacing * (a % n_side), offset + spacing * (a // n_side)], axis=1).astype(np.float64)


def check_field(G, pos, re, im, N):
    """G [P][N][N]: each antenna's anchor cell holds its decoded voltage, every other cell 0."""
    x = np.floor(pos[:, 0] + 0.5).astype(int) % N
    y = np.floor(pos[:, 1] + 0.5).astype(int) % N
    got = G[y, x]
    np.testing.assert_array_equal(got.real, re.astype(np.float32))
    np.testing.assert_array_equal(got.imag, im.astype(np.float32))
    mask = np.ones((N, N), bool)
    mask[y, x] = False
    assert (G[mask] == 0).all()


def check_golden(codes, got):
    """The hand-decoded table's rows, looked up among the 256 results."""
    rows = read_golden("unpack_4bit.txt")
    for r in rows:
        i = int(np.nonzero(codes == int(r[0], 16))[0][0])
        assert got[i] == complex(int(r[1]), int(r[2])), r


@pytest.mark.parametrize("P", [1, 2])
def test_fp32_gridding_decodes_every_code_exactly(P):
    codes, re, im = all_codes()
    N = 32
    pos = lattice(16, 2.0)
    volt = np.zeros((1, 1, 256, P), dtype=np.uint8)
    volt[0, 0, :, 0] = codes
    if P == 2:
        volt[0, 0, :, 1] = codes[::-1]
    with moff.Plan(pos, np.ones((256, P, 1, 1)), N, 1, P) as pl:
        G = pl.grid_snapshot(volt, 0)
    check_field(G[0], pos, re, im, N)
    if P == 2:
        check_field(G[1], pos, re[::-1], im[::-1], N)
    x, y = (pos[:, 0]).astype(int), (pos[:, 1]).astype(int)
    check_golden(codes, G[0][y, x].astype(np.complex128))


def test_dft_route_gridding_decodes_every_code_exactly(monkeypatch):
    """A plan on the factored-DFT route grids with the same decode (FP32)."""
    monkeypatch.setenv("MOFF_TC_DFT", "1")
    codes, re, im = all_codes()
    N = 256
    pos = lattice(16, 2.0, offset=100.0)
    volt = codes.reshape(1, 1, 256, 1)
    with moff.Plan(pos, np.ones((256, 1, 1, 1)), N, 1, 1, fp16tc=True) as pl:
        assert pl.route() in ("fp16_dft", "fp16_tcgrid")
        G = pl.grid_snapshot(volt, 0)
    check_field(G[0], pos, re, im, N)


def test_fp16_voltage_planes_decode_every_code_exactly():
    codes, re, im = all_codes()
    N, P = 32, 2
    pos = lattice(16, 2.0)
    volt = np.zeros((3, 1, 256, P), dtype=np.uint8)
    for t in range(3):                       # every sample and pol holds a different permutation
        volt[t, 0, :, 0] = np.roll(codes, 17 * t)
        volt[t, 0, :, 1] = np.roll(codes[::-1], 5 * t)
    with moff.Plan(pos, np.ones((256, P, 1, 1)), N, 1, P, fp16tc=True) as pl:
        assert pl.route() == "fp16_rowspec"
        planes, scale = pl.voltage_planes(volt, 0)
    # unit gains: scale 2^e with 16 |g| 2^e in [2^13, 2^14), i.e. 2^9
    assert scale == 512.0
    z = planes / scale
    want_re = np.stack([np.roll(re, 17 * t) for t in range(3)]), np.stack([np.roll(re[::-1], 5 * t) for t in range(3)])
    want_im = np.stack([np.roll(im, 17 * t) for t in range(3)]), np.stack([np.roll(im[::-1], 5 * t) for t in range(3)])
    for q in range(P):
        np.testing.assert_array_equal(z[:, :, q].real, want_re[q])
        np.testing.assert_array_equal(z[:, :, q].imag, want_im[q])
    check_golden(codes, z[0, :, 0].astype(np.complex128))


def test_read_image_timeout_leaves_plan_unchanged():
    cfg = synth.config_dualpol()
    A, P, C, N, T = cfg["pos"].shape[0], 2, cfg["n_chan"], cfg["grid_n"], 128
    codes = synth.device_codes(8123669 + 303, T, C, A, P)

    def run(poll_first):
        with moff.Plan(cfg["pos"], cfg["taps"], N, C, P) as pl:
            pl.set_gains(cfg["gains"])
            for _ in range(3):                # about 60 ms of queued work
                pl.submit(codes)
            if poll_first:
                with pytest.raises(moff.MoffError) as e:
                    pl.read_image(timeout_ms=0)
                assert e.value.status == -5
            img, n = pl.read_image()
        return img, n

    ref, n_ref = run(False)
    img, n = run(True)
    assert n == n_ref == 3 * T
    np.testing.assert_array_equal(img, ref)


@pytest.mark.parametrize("shuffle", [False, True])
def test_tcgrid_voltage_planes_decode_exactly_for_large_arrays(shuffle):
    """The plane kernel of large arrays (one thread per plane row) on the tensor-core gridding
    route: warps whose rows hold consecutive voltages read them as aligned 16-byte pieces (a
    lattice in index order), other warps byte by byte (the same lattice with its antennas
    shuffled); rows copied for kernel windows that wrap the grid edge must equal their originals.
    With unit gains every plane value is the decoded voltage times the channel's
    power-of-two scale, exactly, in every sample, also where a 32-sample slice is ragged."""
    rng = np.random.default_rng(404)
    side, N, K, P, C, T = 80, 512, 5, 2, 2, 45
    # the lattice straddles the grid's x edge, so kernel windows wrap and rows are copied
    pos = synth.positions_lattice(rng, side, side, 1.0, 0.05, (N - side, N / 2 - side))
    if shuffle:
        pos = pos[rng.permutation(len(pos))]
    A = len(pos)
    taps = synth.taps_gaussian(rng, pos, K, 1.2, n_pol=P).astype(np.complex64)
    re = rng.integers(-8, 8, size=(T, C, A, P))
    im = rng.integers(-8, 8, size=(T, C, A, P))
    volt = synth.pack_4bit(re, im)
    with moff.Plan(pos, taps, N, C, P, fp16tc=True) as pl:
        assert pl.route() == "fp16_tcgrid"
        pl.set_gains(np.ones((C, A, P), dtype=np.complex64))
        for chan in range(C):
            planes, scale = pl.voltage_planes(volt, chan)
            assert scale == 512.0
            z = planes / scale
            np.testing.assert_array_equal(z.real, re[:, chan])
            np.testing.assert_array_equal(z.imag, im[:, chan])
