"""Host arithmetic of the benchmark line (CPU): the algorithmic byte count per
sweep that the roofline fraction divides by, and the workload sizes it is
quoted on (a 27-point coupling on an nx x ny x nz node lattice has
(3nx-2)(3ny-2)(3nz-2) blocks)."""
import json
import types

import numpy as np

from paper_2201_09212_gb300 import scenes


def test_bytes_per_sweep_of_the_terrain_lattice():
    import bench
    N = 128 * 128 * 32
    sc = types.SimpleNamespace(n_nodes=N, n=3 * N, nnzb=(3 * 128 - 2) ** 2 * (3 * 32 - 2),
                               n_c=128 * 128)
    assert sc.nnzb == 13_716_856
    # FP32: blocks + column indices, row pointers, v read, b read, v written,
    # W, contact records (48 B) and lambda (12 B)
    expect = 40 * sc.nnzb + 4 * (N + 1) + 3 * 4 * sc.n + 4 * N + 60 * sc.n_c
    assert bench.algorithmic_bytes_per_sweep(sc) == expect == 572_725_956
    # FP64 values and vectors, 32-bit indices
    expect64 = 76 * sc.nnzb + 4 * (N + 1) + 3 * 8 * sc.n + 8 * N + 60 * sc.n_c
    assert bench.algorithmic_bytes_per_sweep(sc, esz=8) == expect64


def test_lattice_generator_sizes():
    dims = (6, 5, 4)
    sc = scenes.terrain_lattice(dims=dims)
    assert sc.n_nodes == 6 * 5 * 4 and sc.n == 3 * sc.n_nodes
    assert sc.nnzb == 16 * 13 * 10
    assert sc.n_c == 6 * 5                                 # the bottom layer
    assert np.all(np.diff(sc.row_ptr) <= 27)


def test_peak_source(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6693.8}))
    assert bench.peaks() == (6693.8, "measured")
