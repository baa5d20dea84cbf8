"""The oracle's sensitivity runs (not part of the method) and the
conditioning they measure.

kernel_perturb and stage_noise change the oracle's arithmetic by seeded
relative amounts; the long-integration parity tests compare the GPU paths
with the spread these produce.  Pinned here: zero settings leave the oracle
bitwise unchanged, perturbations have the requested size and symmetry, a
short integration is well conditioned, and a long one of the benchmark grid
in its coagulation-fragmentation balance is not.
"""
import numpy as np

from paper_2402_18471_b300 import synth


def test_zero_settings_are_the_plain_oracle(oracle_mod):
    d = synth.column_1x32().subset([0, 7])
    ref = oracle_mod.Oracle(d).step(d.rho0, d.t_span, log_cap=3000)
    o0 = oracle_mod.Oracle(d, kernel_perturb=0.0, stage_noise=0.0, perturb_seed=5)
    assert np.array_equal(o0.step(d.rho0, d.t_span)["rho"], ref["rho"])
    y = oracle_mod.Oracle(d).replay(d.rho0, ref["log"], ref["n_log"])
    assert np.array_equal(o0.replay(d.rho0, ref["log"], ref["n_log"]), y)


def test_kernel_perturbation_size_and_symmetry(oracle_mod):
    d = synth.column_1x32().subset([3])
    K0, _, _ = oracle_mod.Oracle(d).kernel()
    K1, _, _ = oracle_mod.Oracle(d, kernel_perturb=1e-6, perturb_seed=9).kernel()
    r = K1 / K0 - 1
    assert np.abs(r).max() <= 0.5e-6 * (1 + 1e-9) and np.abs(r).max() > 0.4e-6
    # the same factor for (i, j) and (j, i)
    assert np.abs(r[0] - r[0].T).max() < 1e-15
    K2, _, _ = oracle_mod.Oracle(d, kernel_perturb=1e-6, perturb_seed=10).kernel()
    assert not np.array_equal(K1, K2)


def test_stage_noise_moves_a_short_run_by_its_own_size(oracle_mod):
    """1000 yr of the column (growth, no fragmentation balance yet): noise of
    2^-21 on every stage input moves the state by about that much."""
    d = synth.column_1x32().subset([0, 16, 31])
    ref = oracle_mod.Oracle(d).step(d.rho0, d.t_span, log_cap=3000)
    y0, sp = oracle_mod.replay_spread(d, d.rho0, ref["log"], ref["n_log"], stage_noise=2.0 ** -21)
    S = d.rho0.sum(1)[:, None]
    rel = sp / (np.abs(y0) + 1e-10 * S)
    assert 0 < rel.max() < 1e-4


def test_long_balance_run_amplifies_rounding(oracle_mod):
    """Two cells of the 128 x 64 x 100 benchmark grid over 1e4 yr: a 1e-15
    relative change of the kernel, replayed over the same steps, grows to
    more than 1e-8 of some bins (measured ~5e-6): elementwise agreement after
    such a run can only be asked up to this spread."""
    g = synth.grid_128x64()
    d = g.subset([0, 683])
    ref = oracle_mod.Oracle(d).step(d.rho0, d.t_span, log_cap=3000)
    y0, sp = oracle_mod.replay_spread(d, d.rho0, ref["log"], ref["n_log"], kernel_perturb=1e-15)
    S = d.rho0.sum(1)[:, None]
    rel = sp / (np.abs(y0) + 1e-10 * S)
    assert rel.max() > 1e-8
