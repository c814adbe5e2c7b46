"""Seeded synthetic inputs for the MOFF imaging path.

This module draws the *inputs* of the method -- antenna positions, gridding
kernels, complex gains, 4-bit voltages and 8-bit ADC streams -- shaped like the
compact 21 cm arrays the paper targets (Sec. 1, Sec. 7).  It holds none of the
method's arithmetic: no unpacking, calibration, gridding, transform or
squaring.  Both the FP64 oracle and the CUDA library consume what it returns,
which is why it lives in a package of its own.

Conventions shared with the library's C ABI (these are data formats, not
method steps):

* positions ``pos`` are ``float64 [A][2]`` = (x, y) in grid-cell units; a
  cell is half a wavelength.
* taps are ``complex [A][P][K][K]`` (one kernel per antenna and pol) or, for
  Jones kernels, ``complex [A][2][2][K][K]`` indexed ``[a][p_out][p_in][dy][dx]``.
* voltages are bytes ``uint8 [T][C][A][P]`` holding a 4-bit two's-complement
  real part in the high nibble and the imaginary part in the low nibble.
* gains are ``complex [C][A][P]``.
* ADC streams are ``int8 [A][P][S]``.

The sky model follows the paper's antenna voltage model (Eq. Ea): a source at
sky pixel ``theta`` reaches antenna ``a`` with phase ``exp(-2 pi i p_a . theta / N)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng_for", "pack_4bit", "positions_uniform", "positions_hex", "positions_lattice",
    "taps_gaussian", "taps_jones", "gains_random", "voltages", "adc_stream",
    "config_tiny", "config_dualpol", "config_precision", "config_widefield", "device_codes", "device_gains",
    "device_adc",
]

SEED_BASE = 8123669


def rng_for(seed: int) -> np.random.Generator:
    """Counter-based Philox stream for a seed (host side, reproducible across machines)."""
    return np.random.Generator(np.random.Philox(key=seed))


def pack_4bit(re, im) -> np.ndarray:
    """Pack integer (re, im) in [-8, 7] into one byte: re in the high nibble, im in the low."""
    re = np.asarray(re, dtype=np.int64)
    im = np.asarray(im, dtype=np.int64)
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("4-bit components must lie in [-8, 7]")
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)


def _nearest_cell(p):
    # Input-model choice: a kernel is sampled on the cells around the nearest cell.
    return np.floor(np.asarray(p, dtype=np.float64) + 0.5).astype(np.int64)


# --------------------------------------------------------------------------- positions

def positions_uniform(rng, n_ant: int, extent_lambda: float, min_spacing_lambda: float,
                      cell_lambda: float = 0.5, origin_cells: float = 0.0) -> np.ndarray:
    """Dart-throwing uniform layout in a square of side ``extent_lambda``.

    Returns cell units. Rejects draws closer than ``min_spacing_lambda`` to an
    earlier antenna.
    """
    pts = []
    tries = 0
    while len(pts) < n_ant:
        tries += 1
        if tries > 200000:
            raise RuntimeError("dart throwing did not converge")
        p = rng.uniform(0.0, extent_lambda, size=2)
        if pts and np.min(np.hypot(*(np.asarray(pts) - p).T)) < min_spacing_lambda:
            continue
        pts.append(p)
    return np.asarray(pts) / cell_lambda + origin_cells


def positions_hex(rng, n_ant: int, spacing_lambda: float, jitter_frac: float,
                  center_cells, cell_lambda: float = 0.5) -> np.ndarray:
    """The ``n_ant`` hex-lattice points nearest the centre, with Gaussian jitter."""
    m = int(np.ceil(np.sqrt(n_ant))) + 4
    ii, jj = np.meshgrid(np.arange(-m, m + 1), np.arange(-m, m + 1), indexing="xy")
    x = (ii + 0.5 * (jj % 2)) * spacing_lambda
    y = jj * (np.sqrt(3.0) / 2.0) * spacing_lambda
    x = x.ravel(); y = y.ravel()
    order = np.lexsort((x, y, np.hypot(x, y)))[:n_ant]
    pts = np.stack([x[order], y[order]], axis=1)
    pts = pts + rng.normal(0.0, jitter_frac * spacing_lambda, size=pts.shape)
    return pts / cell_lambda + np.asarray(center_cells, dtype=np.float64)


def positions_lattice(rng, nx: int, ny: int, pitch_lambda: float, jitter_frac: float,
                      origin_cells, cell_lambda: float = 0.5) -> np.ndarray:
    """Rectangular ``nx`` x ``ny`` lattice with Gaussian jitter (x fastest)."""
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    pts = np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.float64) * pitch_lambda
    pts = pts + rng.normal(0.0, jitter_frac * pitch_lambda, size=pts.shape)
    return pts / cell_lambda + np.asarray(origin_cells, dtype=np.float64)


# --------------------------------------------------------------------------- kernels

def taps_gaussian(rng, pos, ksize: int, sigma_cells: float, n_pol: int = 1,
                  subpixel: bool = True, phase_slope: float = 0.0,
                  normalise: str = "sum") -> np.ndarray:
    """Per-antenna Gaussian aperture kernels ``complex128 [A][P][K][K]``.

    ``subpixel`` evaluates the Gaussian at (cell - true position); otherwise
    at integer offsets, so every antenna shares one kernel.  ``phase_slope``
    > 0 multiplies each antenna-pol kernel by a seeded smooth phase
    ``exp(i(alpha + beta dx + gamma dy))`` with ``beta, gamma ~ U(-s, s)``.
    """
    pos = np.asarray(pos, dtype=np.float64)
    A = pos.shape[0]
    h = ksize // 2
    d = np.arange(ksize) - h
    anc = _nearest_cell(pos)
    off = (anc - pos) if subpixel else np.zeros_like(pos)          # [A][2]
    dx = d[None, None, :] + off[:, 0, None, None]                  # [A][1][K]
    dy = d[None, :, None] + off[:, 1, None, None]                  # [A][K][1]
    g = np.exp(-(dx ** 2 + dy ** 2) / (2.0 * sigma_cells ** 2))    # [A][K][K]
    if normalise == "sum":
        g = g / g.sum(axis=(1, 2), keepdims=True)
    taps = np.repeat(g[:, None, :, :], n_pol, axis=1).astype(np.complex128)
    if phase_slope > 0.0:
        alpha = rng.uniform(0.0, 2 * np.pi, size=(A, n_pol))
        beta = rng.uniform(-phase_slope, phase_slope, size=(A, n_pol))
        gamma = rng.uniform(-phase_slope, phase_slope, size=(A, n_pol))
        ph = (alpha[:, :, None, None] + beta[:, :, None, None] * d[None, None, None, :]
              + gamma[:, :, None, None] * d[None, None, :, None])
        taps = taps * np.exp(1j * ph)
    return taps


def taps_jones(rng, pos, ksize: int, sigma_cells: float, leak: float = 0.05,
               w_alpha: float = 0.3) -> np.ndarray:
    """2x2 Jones kernels ``complex128 [A][2][2][K][K]`` for the wide-field layout.

    Gaussian beam times ``diag(1 + 0.1 * smooth)`` plus a ``leak`` leakage
    term on the off-diagonals, all times a non-coplanar w-phase
    ``exp(i alpha_a (dx^2 + dy^2))`` with ``alpha_a ~ U(-w_alpha, w_alpha)``.
    """
    pos = np.asarray(pos, dtype=np.float64)
    A = pos.shape[0]
    h = ksize // 2
    d = np.arange(ksize) - h
    anc = _nearest_cell(pos)
    off = anc - pos
    dx = d[None, None, :] + off[:, 0, None, None]
    dy = d[None, :, None] + off[:, 1, None, None]
    g = np.exp(-(dx ** 2 + dy ** 2) / (2.0 * sigma_cells ** 2))
    g = g / g.sum(axis=(1, 2), keepdims=True)
    smooth = rng.uniform(-1.0, 1.0, size=(A, 2, 3))
    s = (smooth[:, :, 0, None, None] + smooth[:, :, 1, None, None] * dx[:, None] / (h + 1)
         + smooth[:, :, 2, None, None] * dy[:, None] / (h + 1))           # [A][2][K][K]
    lk = leak * np.exp(1j * rng.uniform(0, 2 * np.pi, size=(A, 2)))
    alpha = rng.uniform(-w_alpha, w_alpha, size=A)
    wph = np.exp(1j * alpha[:, None, None] * (dx ** 2 + dy ** 2))         # [A][K][K]
    J = np.zeros((A, 2, 2, ksize, ksize), dtype=np.complex128)
    J[:, 0, 0] = g * (1.0 + 0.1 * s[:, 0])
    J[:, 1, 1] = g * (1.0 + 0.1 * s[:, 1])
    J[:, 0, 1] = g * lk[:, 0, None, None]
    J[:, 1, 0] = g * lk[:, 1, None, None]
    return J * wph[:, None, None]


# --------------------------------------------------------------------------- gains, voltages

def gains_random(rng, n_chan: int, n_ant: int, n_pol: int,
                 amp=(0.8, 1.2)) -> np.ndarray:
    """Complex gains ``[C][A][P]`` with amplitude U(amp) and phase U(0, 2 pi)."""
    a = rng.uniform(amp[0], amp[1], size=(n_chan, n_ant, n_pol))
    ph = rng.uniform(0.0, 2 * np.pi, size=(n_chan, n_ant, n_pol))
    return a * np.exp(1j * ph)


def voltages(rng, n_time: int, n_chan: int, pos, n_pol: int, grid_n: int,
             sources=(), noise_sigma: float = 2.0, instr_gains=None,
             source_sigma: float = 1.0):
    """4-bit complex voltages ``uint8 [T][C][A][P]`` (Eq. Ea sky model + noise).

    ``sources`` is a sequence of integer sky pixels (kx, ky).  Each source has
    an independent complex Gaussian amplitude per (t, c, pol) with standard
    deviation ``source_sigma``; antenna ``a`` sees it with phase
    ``exp(-2 pi i (x_a kx + y_a ky) / N)``.  ``instr_gains [C][A][P]``, if
    given, multiply the field before digitisation.  Components are rounded
    and clipped to [-7, 7].  Returns ``(codes, re, im)``.
    """
    pos = np.asarray(pos, dtype=np.float64)
    A = pos.shape[0]
    shape = (n_time, n_chan, A, n_pol)
    v = rng.normal(0.0, noise_sigma, size=shape) + 1j * rng.normal(0.0, noise_sigma, size=shape)
    for (kx, ky) in sources:
        ph = np.exp(-2j * np.pi * (pos[:, 0] * kx + pos[:, 1] * ky) / grid_n)      # [A]
        amp = (rng.normal(0.0, source_sigma / np.sqrt(2), size=(n_time, n_chan, 1, n_pol))
               + 1j * rng.normal(0.0, source_sigma / np.sqrt(2), size=(n_time, n_chan, 1, n_pol)))
        v = v + amp * ph[None, None, :, None]
    if instr_gains is not None:
        v = v * np.asarray(instr_gains)[None]
    re = np.clip(np.rint(v.real), -7, 7).astype(np.int64)
    im = np.clip(np.rint(v.imag), -7, 7).astype(np.int64)
    return pack_4bit(re, im), re, im


def adc_stream(rng, n_ant: int, n_pol: int, n_samp: int, sigma: float = 20.0,
               tones=()) -> np.ndarray:
    """8-bit real ADC samples ``int8 [A][P][S]``: Gaussian noise plus tones.

    ``tones`` is a sequence of ``(cycles_per_sample, amplitude)``; each antenna
    gets a seeded random phase per tone.
    """
    x = rng.normal(0.0, sigma, size=(n_ant, n_pol, n_samp))
    n = np.arange(n_samp)
    for (f, amp) in tones:
        ph = rng.uniform(0, 2 * np.pi, size=(n_ant, n_pol, 1))
        x = x + amp * np.cos(2 * np.pi * f * n[None, None, :] + ph)
    return np.clip(np.rint(x), -127, 127).astype(np.int8)


# --------------------------------------------------------------------------- workloads

def config_tiny(seed: int = SEED_BASE + 0, n_time: int = 256, n_chan: int = 16):
    """Plain MOFF, tiny: 64 antennas uniform in 16x16 lambda (>= 1 lambda apart),
    single pol, 16 channels, 256 samples, N=32, one shared 3x3 real Gaussian
    kernel, noise sigma 2 plus 3 point sources, gains |g| ~ U(0.8, 1.2)."""
    rng = rng_for(seed)
    N = 32
    pos = positions_uniform(rng, 64, 16.0, 1.0)
    taps = taps_gaussian(rng, pos, 3, 0.5, n_pol=1, subpixel=False)
    srcs = [tuple(int(v) for v in rng.integers(0, N, size=2)) for _ in range(3)]
    codes, _, _ = voltages(rng, n_time, n_chan, pos, 1, N, sources=srcs, noise_sigma=2.0)
    gains = gains_random(rng, n_chan, 64, 1)
    return dict(pos=pos, taps=taps, grid_n=N, n_chan=n_chan, n_pol=1, codes=codes,
                gains=gains, sources=srcs, jones=False)


def config_dualpol(seed: int = SEED_BASE + 1, n_ant: int = 1024, grid_n: int = 128,
                   n_chan: int = 1024, ksize: int = 7):
    """Dual-pol array: hex-packed core at 1.5 lambda spacing with 5 % jitter,
    7x7 complex kernels (Gaussian sigma 1.2 cells times a seeded smooth phase).
    Returns the array description; voltages or ADC are drawn separately."""
    rng = rng_for(seed)
    c = grid_n / 2.0
    pos = positions_hex(rng, n_ant, 1.5, 0.05, (c, c))
    taps = taps_gaussian(rng, pos, ksize, 1.2, n_pol=2, subpixel=True, phase_slope=0.3)
    gains = gains_random(rng, n_chan, n_ant, 2)
    return dict(pos=pos, taps=taps, grid_n=grid_n, n_chan=n_chan, n_pol=2, gains=gains,
                jones=False, rng=rng)


def config_precision(seed: int = SEED_BASE + 2, side: int = 128, grid_n: int = 512,
                     n_chan: int = 1024, ksize: int = 7, with_gains: bool = True):
    """Filled aperture: side x side antennas on a 1 lambda lattice (5 % jitter),
    dual pol, 7x7 kernels, in the centre of a grid zero-padded by two.
    ``with_gains=False`` skips the host gains (draw them with ``device_gains``)."""
    rng = rng_for(seed)
    o = grid_n / 2.0 - side          # lattice spans 2*side cells, centred
    pos = positions_lattice(rng, side, side, 1.0, 0.05, (o, o))
    taps = taps_gaussian(rng, pos, ksize, 1.2, n_pol=2, subpixel=True, phase_slope=0.3)
    gains = gains_random(rng, n_chan, pos.shape[0], 2) if with_gains else None
    return dict(pos=pos, taps=taps, grid_n=grid_n, n_chan=n_chan, n_pol=2, gains=gains,
                jones=False, rng=rng)


def config_widefield(seed: int = SEED_BASE + 4, nx: int = 256, ny: int = 128, grid_n: int = 512,
                     n_chan: int = 4096, ksize: int = 9, with_gains: bool = True):
    """Wide-field: nx x ny antennas at 1 lambda pitch (x wraps the grid), full
    pol with 9x9 Jones kernels carrying a w-phase.  ``with_gains=False`` skips
    the host gains (draw them with ``device_gains``)."""
    rng = rng_for(seed)
    pos = positions_lattice(rng, nx, ny, 1.0, 0.05, (0.0, grid_n / 2.0 - ny))
    taps = taps_jones(rng, pos, ksize, 1.5)
    gains = gains_random(rng, n_chan, pos.shape[0], 2) if with_gains else None
    return dict(pos=pos, taps=taps, grid_n=grid_n, n_chan=n_chan, n_pol=2, gains=gains,
                jones=True, rng=rng)


# --------------------------------------------------------------------------- device-side draws (large workloads)

def config_serving(seed: int = SEED_BASE + 3, n_arrays: int = 8, chans=(64, 128, 256, 512, 1024),
                   t_range=(100, 1000), ksize: int = 7):
    """Sub-arrays of uneven size for a request stream: A drawn from {256, 1024,
    4096, 16384} on a square 1 lambda lattice (ceil(sqrt A) per side, 5 % jitter)
    centred in a grid N drawn from {64, 128, 256, 512} with N >= 2 ceil(sqrt A)
    cells, dual pol, 7x7 kernels; per array a channel count from ``chans`` (64 to
    1024) and a block length in ``t_range`` (100 to 1000 samples)."""
    rng = rng_for(seed)
    out = []
    for _ in range(n_arrays):
        A = int(rng.choice([256, 1024, 4096, 16384]))
        side = int(np.ceil(np.sqrt(A)))
        N = int(rng.choice([n for n in (64, 128, 256, 512) if n >= 2 * side]))
        C = int(rng.choice(list(chans)))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        o = N / 2.0 - side
        pos = positions_lattice(rng, side, side, 1.0, 0.05, (o, o))[:A]
        taps = taps_gaussian(rng, pos, ksize, 1.2, n_pol=2, subpixel=True, phase_slope=0.3)
        gains = gains_random(rng, C, A, 2)
        out.append(dict(A=A, N=N, C=C, T=T, pos=pos, taps=taps, gains=gains))
    return out


def device_codes(seed: int, n_time: int, n_chan: int, n_ant: int, n_pol: int,
                 sigma: float = 2.0, chunk: int = 32):
    """4-bit voltages ``uint8 [T][C][A][P]`` drawn on the GPU with a seeded torch
    Philox generator: Gaussian noise of ``sigma`` per component, rounded and
    clipped to [-7, 7], packed re-high/im-low.  For workloads too large to draw
    on the host; the values are reproducible for a given seed."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    out = torch.empty((n_time, n_chan, n_ant, n_pol), dtype=torch.uint8, device="cuda")
    # at most ~1 GB of float temporaries per draw (the wide-field block is 268 M voltages per sample)
    chunk = max(1, min(chunk, (1 << 28) // max(1, n_chan * n_ant * n_pol)))
    for t0 in range(0, n_time, chunk):
        n = min(chunk, n_time - t0)
        shape = (n, n_chan, n_ant, n_pol)
        re = torch.clamp(torch.round(torch.randn(shape, generator=g, device="cuda") * sigma), -7, 7).to(torch.int32)
        im = torch.clamp(torch.round(torch.randn(shape, generator=g, device="cuda") * sigma), -7, 7).to(torch.int32)
        out[t0:t0 + n] = (((re & 15) << 4) | (im & 15)).to(torch.uint8)
    return out


def device_gains(seed: int, n_chan: int, n_ant: int, n_pol: int, amp=(0.8, 1.2)):
    """Complex gains ``complex64 [C][A][P]`` drawn on the GPU (seeded torch Philox):
    amplitude U(amp), phase U(0, 2 pi), as ``gains_random`` draws them on the host.
    For channel counts whose gains are too large to draw on the host."""
    import math
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    shape = (n_chan, n_ant, n_pol)
    a = amp[0] + (amp[1] - amp[0]) * torch.rand(shape, generator=g, device="cuda")
    ph = 2 * math.pi * torch.rand(shape, generator=g, device="cuda")
    return torch.polar(a, ph).to(torch.complex64)


def device_adc(seed: int, pos, n_pol: int, n_samp: int, frame: int, grid_n: int,
               sigma: float = 20.0, sources=((40, 70, 100, 12.0), (90, 30, 600, 8.0), (64, 64, 900, 6.0)),
               chunk: int = 32):
    """8-bit real ADC streams ``int8 [A][P][S]`` drawn on the GPU: Gaussian
    noise of ``sigma`` plus narrow-band sky sources.  Each source
    ``(kx, ky, channel, amplitude)`` is a tone at the centre of ``channel``
    (``channel / frame`` cycles per sample) whose phase at antenna ``a`` is
    ``-2 pi (x_a kx + y_a ky) / N`` (the Eq. Ea sky model at that channel)."""
    import math
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    pos_t = torch.as_tensor(np.asarray(pos, dtype=np.float64), device="cuda")
    A = pos_t.shape[0]
    n = torch.arange(n_samp, device="cuda", dtype=torch.int64)
    out = torch.empty((A, n_pol, n_samp), dtype=torch.int8, device="cuda")
    for a0 in range(0, A, chunk):
        a1 = min(A, a0 + chunk)
        x = torch.randn((a1 - a0, n_pol, n_samp), generator=g, device="cuda") * sigma
        for (kx, ky, ch, amp) in sources:
            ph = (-2 * math.pi * (pos_t[a0:a1, 0] * kx + pos_t[a0:a1, 1] * ky) / grid_n).to(torch.float32)
            # tone phase reduced exactly in integers before going to float32
            tone = (2 * math.pi / frame) * ((int(ch) * n) % frame).to(torch.float32)
            x += (amp * torch.cos(tone[None, :] + ph[:, None]))[:, None, :]
        out[a0:a1] = torch.clamp(torch.round(x), -127, 127).to(torch.int8)
    return out
