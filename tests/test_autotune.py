"""Host logic of the autotuner (no GPU): the work-list size model, the
wave-aligned sweep candidates and the temporal-blocking candidates."""
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


def test_band_candidates_fill_their_waves():
    ws = [synth.free_dendrite_2d(1024, 5.0 * t) for t in range(10)]
    resident = 2432
    for base in ((64, 1, 38), (64, 1, 8)):
        cands = A.band_candidates(ws, base, resident)
        assert [c[:4] for c in cands] == [base + (2,)] * len(cands)
        per_row = 10 * 18  # 60-column strips of ten 1024-column instances
        for k, c in zip((1, 2), cands):
            bs = c[4]
            # the fewest sweeps per band whose items fill k waves, at most half the depth
            half = -(-(-(-1024 // base[2])) // 2)
            assert bs == half or (bs * per_row >= k * resident and (bs == 1 or (bs - 1) * per_row < k * resident))
            assert bs <= half
    # 27 sweeps of 38 rows cover the 1024 rows: one band, the depth-1 schedule, is not raced
    assert A.band_candidates(ws, (64, 1, 38), resident) == [(64, 1, 38, 2, 14)]
    assert A.band_candidates(ws, (64, 1, 8), resident) == [(64, 1, 8, 2, 14), (64, 1, 8, 2, 28)]
    # two 256^2 instances cannot fill the GPU with one band: two bands of 16 sweeps
    small = [synth.free_dendrite_2d(256), synth.free_dendrite_2d(256)]
    assert A.band_candidates(small, (64, 1, 8), resident) == [(64, 1, 8, 2, 16)]
    assert A.band_candidates(small, (64, 1, 256), resident) == []  # one sweep: no band to split


def test_split_bands_and_depth_race():
    assert A.split((64, 1, 38)) == ((64, 1, 38), (1, 1))
    assert A.split([34, 10, 8, 2, 3]) == ((34, 10, 8), (2, 3))
    ws = [synth.free_dendrite_2d(1024), synth.free_dendrite_2d(200)]
    assert A.bands(ws, (64, 1, 38)) == 1
    assert A.bands(ws, (64, 1, 8, 2, 14)) == 10  # 128 sweeps of the deeper instance in bands of 14
    w3 = [synth.free_dendrite_3d(64)]
    assert A.bands(w3, (34, 10, 16, 2, 3)) == 2
    r = A.depth_race({"(64, 1, 38)": 1.2e-4, "(64, 1, 8, 2, 14)": 1.6e-4, "(64, 1, 12)": 1.3e-4,
                      "(64, 1, 38, 2, 27)": 1.25e-4})
    assert r["depth1_tile"] == [64, 1, 38] and abs(r["depth1_ms"] - 0.12) < 1e-12
    assert r["depth2_tile"] == [64, 1, 38, 2, 27] and abs(r["depth2_ms"] - 0.125) < 1e-12


def test_wavefront_eligibility():
    w = synth.free_dendrite_2d(64)
    assert A.wavefront_ok(w)
    w.thermal = 1
    assert not A.wavefront_ok(w)
    w.thermal, w.kernels = 0, 1
    assert not A.wavefront_ok(w)
