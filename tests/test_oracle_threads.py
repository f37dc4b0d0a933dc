"""The oracle's OpenMP passes (rows of the stencil passes, the flat per-cell
passes, ghost filling) give bit-identical results on any number of threads:
each cell's arithmetic is independent of the partition."""
import os
import subprocess
import sys

import numpy as np


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = """
import sys, numpy as np
sys.path.insert(0, {root!r})
from oracle import oracle as O
from tests.helpers import small_workload, oracle_params
from paper_2110_12448_gb300 import synth
out = []
for dim, scheme in ((2, "S21"), (2, "SBAR21"), (3, "SBAR120")):
    w = small_workload(dim, 37, 29, 11 if dim == 3 else 1, scheme=scheme)
    rng = np.random.default_rng(4)
    psi, U = synth.random_state(rng, w)
    g, rots = synth.random_grains(rng, w, 3)
    p, u = O.step(oracle_params(w, scheme), rots, g, psi, U, 3)
    out += [p, u]
np.savez({path!r}, *out)
"""


def run(tmp_path, threads):
    path = str(tmp_path / f"t{threads}.npz")
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    subprocess.run([sys.executable, "-c", CODE.format(root=ROOT, path=path)], env=env, cwd=ROOT, check=True,
                   timeout=300)
    with np.load(path) as z:
        return [z[k] for k in sorted(z.files, key=lambda s: int(s.split("_")[1]))]


def test_oracle_bitwise_independent_of_thread_count(tmp_path):
    one = run(tmp_path, 1)
    many = run(tmp_path, max(4, os.cpu_count() or 4))
    assert len(one) == len(many) == 6
    for a, b in zip(one, many):
        assert np.array_equal(a, b)
