"""Host logic of the autotuner (no GPU): the work-list size model and the
wave-aligned sweep candidates."""
from paper_2110_12448_gb300 import autotune as A
from paper_2110_12448_gb300 import synth


def test_work_items_model():
    w = synth.free_dendrite_2d(1024)
    assert A.work_items(w, (64, 1, 40)) == 18 * 26  # 60-column strips x 40-row bands
    assert A.work_items(w, (64, 1, 2048)) == 18
    w3 = synth.free_dendrite_3d(64)
    assert A.work_items(w3, (34, 10, 16)) == 3 * 11 * 4  # 30 x 6 columns x 16-plane bands


def test_wave_aligned_sweeps_are_minimal_for_their_wave_count():
    ws = [synth.free_dendrite_2d(1024, 5.0 * t) for t in range(10)]
    resident = 2432
    cands = A.wave_aligned(ws, 64, 1, resident)
    assert cands and all(t[:2] == (64, 1) for t in cands)
    sweeps = [t[2] for t in cands]
    assert sweeps == sorted(sweeps, reverse=True)
    for sw in sweeps:
        n = sum(A.work_items(w, (64, 1, sw)) for w in ws)
        k = -(-n // resident)
        # fits in k waves, and one row shorter would not
        assert n <= k * resident
        assert sw == 8 or sum(A.work_items(w, (64, 1, sw - 1)) for w in ws) > k * resident
    # ten 1024^2 instances on 2432 warps: 38-row sweeps fill two waves to 99.9 %
    assert 38 in sweeps


def test_wave_aligned_handles_batches_larger_than_one_wave_per_band():
    w3 = [synth.free_dendrite_3d(256)]
    cands = A.wave_aligned(w3, 34, 10, 304)
    assert cands[0][2] == 256  # whole-depth sweeps already need two waves
    assert all(8 <= t[2] <= 256 for t in cands)
