"""Failure detection without a GPU fault: a launch failure injected on the host
(pf_debug_inject_launch_failure) surfaces as PF_ERR_CUDA with its message, the
handle or group advances by exactly the steps that launched (checked against
the oracle), and stepping resumes normally afterwards."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2110_12448_gb300 import synth
from tests.helpers import oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import native as N
    N.lib()
    yield N
    N.inject_launch_failure(-1)


def setup(N, seed, stream=None):
    rng = np.random.default_rng(seed)
    w = synth.free_dendrite_2d(70, ny=33)
    psi, U = synth.random_state(rng, w)
    s = N.Sim.from_workload(w, "f64", stream=stream)
    s.set_fields(psi, U)
    return w, psi, U, s


def check(w, s, psi, U, n):
    gp, gu = s.get_fields()
    op, ou = O.step(oracle_params(w), w.rots, np.zeros(w.shape, np.int16), psi, U, n)
    assert rel_err(gp, op) < max(n, 1) * 1e-12 and rel_err(gu, ou) < max(n, 1) * 1e-12


def test_injected_failure_in_pf_step(native):
    w, psi, U, s = setup(native, 1)
    s.step(4)
    native.inject_launch_failure(3)
    with pytest.raises(native.PfError) as e:
        s.step(10)
    assert e.value.code == native.PF_ERR_CUDA and "injected" in str(e.value)
    assert s.steps_done == 7
    check(w, s, psi, U, 7)
    s.step(5)  # the injection was consumed
    assert s.steps_done == 12
    check(w, s, psi, U, 12)


@pytest.mark.parametrize("use_graph", [False, True])
def test_injected_failure_in_group_step(native, use_graph):
    import torch
    st = torch.cuda.Stream()
    runs = [setup(native, 10 + i, stream=st) for i in range(2)]
    grp = native.Group(2, sum(native.Group.work_items(r[3]) for r in runs), stream=st)
    for r in runs:
        grp.add(r[3])
    native.inject_launch_failure(20)
    with pytest.raises(native.PfError) as e:
        grp.step(40, use_graph=use_graph)
    assert e.value.code == native.PF_ERR_CUDA
    done = 16 if use_graph else 20  # a graph replay of 16 steps fails whole
    for w, psi, U, s in runs:
        assert s.steps_done == done
    grp.step(40 - done, use_graph=use_graph)
    grp.close()
    for w, psi, U, s in runs:
        assert s.steps_done == 40
        check(w, s, psi, U, 40)
