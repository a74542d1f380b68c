"""The bench's CPU baseline leg (the oracle on the host cores, bench.OracleSample): the sample
follows the size the GPU arm solves (--n), reports a measured rate, and only scales to
another size as an explicitly marked estimate. Runs on the CPU with a small mesh."""
import numpy as np

import bench
from oracle import q1
from workload import WORKLOADS, load_sequence, workload_mesh


def test_sample_is_the_workload_when_sizes_match():
    wl = WORKLOADS["graded128"]
    smp = bench.OracleSample("graded128", wl, 16, n=16)
    assert smp.is_full and smp.n_full == 16 and smp.extrapolation(0.1) is None
    t, xs = smp.run(2, start=3)
    assert t > 0 and sorted(xs) == [3, 4]
    mesh = workload_mesh("graded128", n=16)
    K = q1.assemble(mesh)
    F = load_sequence(mesh, wl["seed"], 2, 3)
    for i, step in enumerate((3, 4)):
        r = np.linalg.norm(F[i] - K @ xs[step]) / np.linalg.norm(F[i])
        assert r <= 1e-10, (step, r)
    m = smp.measured(2, t)
    assert m["n"] == 16 and m["solve_steps"] == 2 and m["nnz_L"] > 0


def test_smaller_sample_is_scaled_only_as_a_marked_estimate():
    wl = WORKLOADS["graded128"]
    smp = bench.OracleSample("graded128", wl, 16, n=24)
    assert not smp.is_full and smp.n_full == 24 and smp.sample_n == 16
    ext = smp.extrapolation(0.01)
    assert ext["kind"] == "estimate, not measured"
    assert smp.scale > 1.0 and abs(ext["solves_per_s"] - 1.0 / (0.01 * smp.scale)) < 1e-12
