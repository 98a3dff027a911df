"""Conventions fixed by numbers the paper prints (tests/golden/paper_printed_values.txt)."""
import os

import numpy as np

import oracle
from oracle import OracleConfig

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_printed_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_mesh_cell_is_complex_double():
    """Table 3: the mesh sizes imply 16 bytes (complex FP64) per cell, as the oracle stores."""
    g = _golden()
    cfg = OracleConfig(8, 0.1, 1, -1.0, 1.0, 3)
    plane = oracle.grid(cfg, [0.0], [0.0], [0.0], np.array([1.0], np.complex64))
    cell_bytes = plane.itemsize
    for nu, nw, gb in [("medium_mesh_nu", "medium_mesh_nw", "medium_mesh_gb"),
                       ("large_mesh_nu", "large_mesh_nw", "large_mesh_gb")]:
        total = g[nu] ** 2 * g[nw] * cell_bytes / 2**30
        assert abs(total - g[gb]) < 1e-9


def test_grid_point_additions_count_taps():
    """Section 4.2: grid-point additions = N_vis x W^2 (26.65e9 for ~0.54e9 visibilities, W=7).

    The oracle's footprint has exactly W x W taps per visibility.
    """
    g = _golden()
    W = int(g["kernel_support"])
    implied = g["medium_grid_point_additions"] / W**2
    assert abs(implied - g["medium_n_vis"]) / g["medium_n_vis"] < 0.01  # "approx" 0.54e9
    cfg = OracleConfig(64, 0.1, 1, -1.0, 1.0, W)
    plane = oracle.grid(cfg, [13.0], [-7.0], [0.0], np.array([1.0], np.complex64))[0]
    assert np.count_nonzero(plane) == W * W
