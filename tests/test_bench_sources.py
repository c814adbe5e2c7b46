"""Host-side parts of the benchmark.  It reports a kernel's DRAM traffic only
while the kernel's source is the one the ncu capture ran: check that every
hashed region is found in its file (a missing marker would silently hash the
whole file) and that every recorded capture names a kernel the benchmark
hashes.  And the algorithmic byte model of the tensor-core row contraction."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_hashed_regions_exist_and_are_nonempty():
    for key, src in bench.KERNEL_SOURCES.items():
        for f in src:
            if isinstance(f, str):
                assert os.path.isfile(os.path.join(ROOT, f)), (key, f)
                continue
            path, start, end = (f[0], None, f[1]) if len(f) == 2 else f
            text = open(os.path.join(ROOT, path)).read()
            i = 0
            if start is not None:
                i = text.find(start)
                assert i >= 0, (key, "start marker missing", start)
            j = text.find(end, i)
            assert j > i, (key, "end marker missing or before start", end)
        assert len(bench.source_sha1(src)) == 40


def test_recorded_captures_name_hashed_kernels():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, r in rec.items():
        kernel = name.split("@")[0]
        assert kernel in bench.KERNEL_SOURCES, name
        assert r.get("bytes_per_launch", r.get("bytes_per_unit", 0)) > 0 and len(r["source_sha1"]) == 40
        assert os.path.exists(os.path.join(ROOT, r["from"].split()[0])), r["from"]
        # a different region never matches the recorded hash
        assert bench.source_sha1(["include/moff.h"]) != r["source_sha1"]


def test_traffic_scales_per_unit_records(tmp_path, monkeypatch):
    """A record in bytes per unit gives bytes per launch for the launch's units;
    a stale source hash gives nothing."""
    rec = {"k@w": {"bytes_per_unit": 1000, "source_sha1": bench.source_sha1(["include/moff.h"]), "from": "x"},
           "s@w": {"bytes_per_unit": 1000, "source_sha1": "0" * 40, "from": "x"}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "include").mkdir()
    (tmp_path / "include" / "moff.h").write_bytes(open(os.path.join(ROOT, "include", "moff.h"), "rb").read())
    assert bench.traffic_for("k@w", ["include/moff.h"], 7680) == 7680000
    assert bench.traffic_for("k@w", ["include/moff.h"]) is None
    assert bench.traffic_for("s@w", ["include/moff.h"], 7680) is None


def test_row_contraction_byte_model():
    """Rows reached by some kernel row (anchor rows +- K//2, cyclic) times the
    half2 row, plus the FP16 real and imaginary voltage planes."""
    import numpy as np
    pos = np.array([[3.2, 5.4], [9.0, 6.0], [1.0, 12.49]])      # anchor rows 5, 6, 12
    assert bench.tc_row_bytes_per_snapshot(pos, N=16, P=2, K=3) == 2 * 7 * 16 * 4 + 3 * 2 * 2 * 2
    wrap = np.array([[0.0, 15.6]])                                # anchor row 16 -> 0: rows 15, 0, 1
    assert bench.tc_row_bytes_per_snapshot(wrap, N=16, P=1, K=3) == 1 * 3 * 16 * 4 + 1 * 1 * 2 * 2


def test_dense_work_model():
    """Method's work per snapshot of the dense routes on a hand-countable array:
    two antennas with 3x3 one-pol kernels on a 256 grid, anchor rows 10 and 11."""
    import numpy as np
    pos = np.array([[5.0, 10.0], [40.2, 11.4]])
    taps = np.ones((2, 1, 3, 3), dtype=complex)
    taps[1, 0, 0, 0] = 0                                 # 17 nonzero taps
    assert bench.reached_rows(pos, 256, 3) == 4          # rows 9-12
    w = bench.dense_work("fp16_dft", pos, taps, 256, 1, Tb=64)
    fac = 8 * 256 * (16 + 16)
    assert w["grid_rows"]["alu"] == 8 * 17 + 6 * 2
    assert w["grid_rows"]["tensor"] == 4 * fac
    assert w["cols_integrate"]["tensor"] == 256 * fac
    assert w["grid_rows"]["bytes"] == 2 + 4 * 256 * 4
    assert w["cols_integrate"]["bytes"] == 4 * 256 * 4 + 2 * 256 * 256 * 8 / 64
    w32 = bench.dense_work("fp32", pos, taps, 256, 1, Tb=64)
    assert w32["grid_rows"]["alu"] == 8 * 17 + 6 * 2 + 4 * 5 * 256 * 8
    assert w32["cols_integrate"]["bytes"] == 4 * 256 * 8 + 2 * 256 * 256 * 8 / 64


def test_tcgrid_work_model():
    """The tensor-core gridding route's kernels: taps' flops for the gridding, the
    factored DFT for both transform axes, the FP16 field written once and read once
    between each pair of kernels."""
    import numpy as np
    pos = np.array([[5.0, 10.0], [7.0, 20.0]])           # anchors (5, 10), (7, 20); 3x3 kernels
    taps = np.ones((2, 1, 3, 3), dtype=complex)
    taps[1] = 0                                          # the second antenna contributes no taps ...
    # ... but still reaches cells: rows 9-11 x columns 4-6 (tile (1, 0)); rows 19-21 x columns 6-8
    # (tiles (2, 0) and (2, 1))
    assert bench.active_tiles(pos, 256, 3) == 3
    w = bench.dense_work("fp16_tcgrid", pos, taps, 256, 1, Tb=128)
    fac = 8 * 256 * 32
    assert w["grid_rows"]["tensor"] == 8 * 9
    assert w["row_transform"]["tensor"] == 6 * fac and w["cols_integrate"]["tensor"] == 256 * fac
    assert w["row_transform"]["bytes"] == 3 * 64 * 4 + 6 * 256 * 4
