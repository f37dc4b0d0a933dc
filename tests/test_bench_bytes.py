"""Algorithmic bytes per cell update of the bench's roofline (no GPU): the
state (psi, U read and written) plus the int16 grain index where the step
reads it, in 3D always and in 2D only for instances with cells outside
grain 0."""
import numpy as np

import bench
from paper_2110_12448_gb300 import synth


def test_one_grain_2d_reads_no_grain_index():
    ws = synth.orientation_sweep_2d(64)
    assert all(int(max(w.seed_grain)) == 0 for w in ws)
    assert bench.bytes_per_cell(ws, "f32") == 16
    assert bench.bytes_per_cell(ws, "f64") == 32
    assert bench.bytes_per_cell(ws, "f32c") == 32
    assert bench.bytes_per_cell(ws, "f32", two=True) == 32


def test_polycrystals_and_3d_read_the_grain_index():
    poly = synth.polycrystal_batch_2d(4, lo=64, hi=96)
    assert all(int(max(w.seed_grain)) > 0 for w in poly)
    assert bench.bytes_per_cell(poly, "f32") == 18
    assert bench.bytes_per_cell([synth.free_dendrite_3d(32)], "f32") == 18


def test_mixed_batch_weights_by_cells():
    one = synth.free_dendrite_2d(64)                       # 4096 cells, grain 0 only
    poly = synth.polycrystal_2d(np.random.default_rng(1), 128, 3)  # 16384 cells, three grains
    b = bench.bytes_per_cell([one, poly], "f32")
    assert abs(b - (16 + 2 * 16384 / (4096 + 16384))) < 1e-12
