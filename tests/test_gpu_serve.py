"""Serving loop on the GPU: continuous batching of mixed 2D/3D requests that
arrive while others run.  Each result must equal the same run stepped alone
(same kernel, same tiling, same per-cell arithmetic): bitwise."""
import numpy as np
import pytest

from paper_2110_12448_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    return N


@pytest.mark.parametrize("n_streams", [1, 2, 3])
def test_served_results_equal_alone(native, n_streams):
    from paper_2110_12448_gb300.serve import Request, Server
    rng = np.random.default_rng(31)
    reqs = []
    for i in range(7):
        if i % 3 == 2:
            w = synth.polycrystal_3d(rng, int(rng.integers(20, 36)), int(rng.integers(1, 4)))
        else:
            w = synth.polycrystal_2d(rng, int(rng.integers(60, 200)), int(rng.integers(1, 5)),
                                     U0=float(rng.uniform(-0.7, -0.4)))
        prec = "f64" if i == 4 else "f32"
        reqs.append(Request(i, w, steps=int(rng.integers(20, 120)), precision=prec, arrival_s=0.02 * i,
                            keep_fields=True))
    srv = Server(chunk=16, budget_bytes=1 << 30, n_streams=n_streams)
    res = {r.rid: r for r in srv.run(reqs)}
    summ = srv.summary()
    srv.close()
    assert len(res) == len(reqs)
    assert summ["p99_s"] >= summ["p50_s"] > 0
    for r in reqs:
        s = native.Sim.from_workload(r.workload, r.precision)
        s.step(r.steps)
        psi, U = s.get_fields()
        got = res[r.rid]
        assert got.obs["step"] == r.steps
        assert np.array_equal(got.fields[0], psi) and np.array_equal(got.fields[1], U), r.rid
        s.close()


def test_budget_limits_concurrency(native):
    from paper_2110_12448_gb300.serve import Request, Server
    ws = [synth.free_dendrite_2d(128, theta_deg=5.0 * i) for i in range(4)]
    one = native.required_bytes(native.make_params(2, 128, 128, max_grains=1, max_seeds=1))
    srv = Server(chunk=8, budget_bytes=2 * one + 1)
    reqs = [Request(i, w, steps=24) for i, w in enumerate(ws)]
    res = srv.run(reqs)
    srv.close()
    assert len(res) == 4
    # at most two ran at once: the last two were admitted only after earlier ones finished
    admits = sorted(r.admit_s for r in res)
    dones = sorted(r.done_s for r in res)
    assert admits[2] >= dones[0] - 1e-6


def test_autotuner_picks_a_valid_tile(native):
    from paper_2110_12448_gb300 import autotune
    ws = [synth.free_dendrite_2d(256, theta_deg=t) for t in (0.0, 10.0)]
    tile, times = autotune.tune(ws, "f32", steps=8, repeats=1, use_cache=False)
    timed = {tuple(int(x) for x in k.strip("()").split(",")): t for k, t in times.items()}
    # every fixed candidate is timed, the extra ones are wave-aligned sweeps,
    # and the answer is the fastest
    assert set(autotune.CANDIDATES_2D) <= set(timed)
    assert all(t[:2] == (64, 1) and t[2] >= 8 for t in timed)
    # the temporal-blocking depth is raced too: depth-2 band wavefronts
    assert any(len(t) == 5 and t[3] == 2 and t[4] >= 1 for t in timed)
    assert tile in timed and timed[tile] == min(timed.values())
    w3 = [synth.free_dendrite_3d(40)]
    tile3, times3 = autotune.tune(w3, "f32", steps=4, repeats=1, use_cache=False)
    timed3 = {tuple(int(x) for x in k.strip("()").split(",")): t for k, t in times3.items()}
    assert tile3 in timed3 and timed3[tile3] == min(timed3.values())
    assert all(t[:2] in {c[:2] for c in autotune.CANDIDATES_3D} for t in timed3)
