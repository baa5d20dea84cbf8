"""The seeded input generator: the MRN start never divides by zero, and the
workloads' seeds select distinct perturbations while the default seed
reproduces the named workload."""
import numpy as np

from paper_2402_18471_b300 import synth


def test_mrn_start_on_a_grid_above_the_cut():
    # every bin above a_cut: all the dust starts in bin 0, no NaN
    a = np.geomspace(1e-3, 1e-1, 6)
    rho = synth.mrn_initial(a, np.array([1e-12, 2e-12]))
    assert np.all(np.isfinite(rho))
    assert np.allclose(rho[:, 0], 0.01 * np.array([1e-12, 2e-12]), rtol=1e-15, atol=0)
    assert np.all(rho[:, 1:] == 0.0)


def test_mrn_start_weights():
    a = np.geomspace(1e-5, 1e-3, 9)
    rho = synth.mrn_initial(a, np.array([1.0]))
    w = np.where(a <= 1e-4 * (1 + 1e-12), np.sqrt(a), 0.0)
    assert np.allclose(rho[0], 0.01 * w / w.sum(), rtol=1e-14, atol=0)


def test_workload_seeds():
    a = synth.grid_128x64()
    b = synth.grid_128x64(seed=1)
    c = synth.grid_128x64(seed=1001)
    assert np.array_equal(a.rho_gas, b.rho_gas)
    assert not np.array_equal(a.rho_gas, c.rho_gas)
