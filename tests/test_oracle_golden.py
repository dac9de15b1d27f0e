"""Pins against numbers the paper prints (tests/golden/table1_benchmarks.txt,
Table 1): the definition G = v / (f h) used for the per-row weight selection
and the "PML nodes inside the grid" reading of the grid sizes."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_benchmarks.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        out.append((t[0],) + tuple(float(x) for x in t[1:]))
    return out


def test_g_range_matches_table1():
    for name, ndof, cm, cM, f, h, Gm, GM, nx, ny, nz in _rows():
        # G = lambda / h = v / (f h), printed to 1-3 significant digits
        assert abs(cm / (f * h) - Gm) <= 0.05 * Gm + 0.05, name
        assert abs(cM / (f * h) - GM) <= 0.01 * GM + 0.05, name


def test_ndof_matches_grid_with_pml_inside():
    for name, ndof, *_rest, nx, ny, nz in _rows():
        if name == "overthrust":     # the paper's own numbers disagree
            continue
        assert abs(nx * ny * nz / 1e6 - ndof) < 0.06, name


def test_homogeneous_grid_is_domain_plus_16_pml_nodes():
    # 10 x 20 x 10 km at h = 50 m: 201 x 401 x 201 nodes, + 2 x 16 PML nodes.
    n = [int(L / 50) + 1 + 2 * 16 for L in (10000, 20000, 10000)]
    assert n == [233, 433, 233]
    assert np.isclose(np.prod(n) / 1e6, 23.5, atol=0.01)
