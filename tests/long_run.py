"""The bound used by the long-integration parity tests.

After thousands of steps in a coagulation-fragmentation balance, the
explicit Bogacki-Shampine integrator run at the paper's tolerance sits near
its stability limit, and right-hand-side differences that vary from one
evaluation to the next grow from step to step: the FP64 oracle itself,
replaying the same steps with its kernel changed by 1e-15 relative, moves
some bins by up to ~1e-5 of themselves (1e-4 on the ring discs).  A GPU
path is held there to what the oracle does when its own arithmetic is
perturbed at that path's level, on top of the strict bound.
"""
import numpy as np


def long_run_bound(oracle_mod, d, rho0, hs, n, precision):
    """Per-bin bound on |GPU - oracle replay of the GPU's accepted steps|:
    1e-5 |rho| + 1e-10 S plus three times the largest deviation of six
    oracle replays perturbed at the path's arithmetic level (FP64: the
    kernel by 1e-15 relative; mixed: every stage input by 2^-21 relative,
    the error bound of the TF32 hi/lo operand split).  Returns the oracle's
    unperturbed replay, the strict bound and the full bound."""
    seeds = (1, 2, 3, 4, 5, 6)
    if precision == "fp64":
        y0, sp = oracle_mod.replay_spread(d, rho0, hs, n, kernel_perturb=1e-15, seeds=seeds)
    else:
        y0, sp = oracle_mod.replay_spread(d, rho0, hs, n, stage_noise=2.0 ** -21, seeds=seeds)
    strict = 1e-5 * np.abs(y0) + 1e-10 * rho0.sum(1)[:, None]
    return y0, strict, strict + 3.0 * sp
