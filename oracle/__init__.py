"""FP64 CPU oracle of the MOFF imaging path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never calls it and shares no
code with it; the two meet only on the seeded inputs drawn by ``synth``.

Parity status per function (what pins it other than itself):

* ``unpack_4bit``      -- hand-decoded byte fixtures and the pack/unpack bijection.
* ``anchors``          -- hand-computed fixtures (half-cell ties round up).
* ``grid_matrix`` / ``grid`` -- brute-force FX identity (Eqs. m1-m6, Bdef),
                          Parseval with non-overlapping footprints, shift invariance.
* ``sky_transform``    -- naive DFT on tiny grids, point-source closed form (sign).
* ``integrate``        -- FX identity (conjugation order of XY), Cauchy-Schwarz,
                          polarisation-scaled inputs.
* ``moff_image``       -- all of the above composed; edge padding (a grid twice as
                          large, footprints not wrapping) samples the same image at
                          every second pixel.
* ``moff_image_sets``  -- a point source imaged through frequency-scaled
                          positions peaks at the same pixel with the closed-form
                          value in every channel; one set equals ``moff_image``.
* ``fx_image``         -- agreement with ``moff_image`` (independent formulation),
                          single-antenna flat image; with ``autos=False`` the
                          baselines-only image equals ``moff_image`` minus ``auto_image``.
* ``auto_image``       -- the same identity; a single delta-kernel antenna gives a
                          flat image of its power.
* ``pfb_window``       -- the 8 coefficients of a 2-tap, M = 4 window against closed
                          forms worked by hand; symmetry; tone-in-bin power.
* ``pfb_spectra``      -- 1-tap rectangular case equals a library FFT, a hand-summed
                          2-tap case, tone-in-bin power.
* ``quantise_4bit``    -- hand fixtures including half-to-even ties and clipping.
* ``antenna_beam`` / ``feedback_sums`` -- the antenna shares sum to the image pixel
                          (FBeq1 = sum over antennas of FBeq2), FBeq3 by brute force
                          over antenna pairs, the point-source closed form.
* ``feedback_delta``   -- zero for a calibrated point-source array; a simulated
                          gain error shrinks to second order in one step with the
                          N reading, while the printed 2N and the unconjugated
                          ratio do not converge.
"""
from .moff_oracle import *  # noqa: F401,F403
