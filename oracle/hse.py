"""hse.py -- plain FP64 CPU oracle of the hydrostatic-equilibrium gas
density of Sec. 3.5 (Eqs. hydroeqbm, hedisc, avcs, heprod, rhonorm) of
Robinson, Booth & Owen, "Introducing cuDisc" (arXiv 2402.18471).

TEST INFRASTRUCTURE.  Only the tests, __graft_entry__.smoke() and bench.py's
CPU-baseline legs use it; it shares no code with the CUDA library.

Per column i of an (R, Z) grid, following the paper's steps in order:
  1. isothermal sound speed c_s^2 = k_B T / (mu m_H) and spherical radius
     r = sqrt(R^2 + Z^2) of every cell;
  2. the pressure ratio of neighbouring cells (Eq. hedisc), with the mean
     reciprocal sound speed squared of the two (Eq. avcs):
       P_j / P_{j-1} = exp[G M_* <1/c_s^2>_j (1/r_j - 1/r_{j-1})];
  3. the pressure relative to cell j = 0 as the running product of those
     ratios (Eq. heprod), which keeps it positive;
  4. the unnormalised density omega_j = (P_j / P_0) / c_s,j^2 (ideal gas);
  5. the normalisation to the column's surface density (Eq. rhonorm):
       rho_j = Sigma_g (R dR) / (sum_k omega_k V_k) omega_j,
     with (R dR) = ((R^e_{i+1})^2 - (R^e_i)^2) / 2 and V_k the cell volumes.
Parity: pinned (isothermal columns telescope to exp[G M_*/c_s^2 (1/r_j -
1/r_0)]; with 1/c_s^2 linear in 1/r the mean of Eq. avcs integrates exactly;
the normalisation; the thin-disc Gaussian limit).
"""
from __future__ import annotations

import math

import numpy as np


def hse_rho_gas(R, Z, T, V, R_edges, Sigma_g, mu, m_H, k_B, GM):
    """Gas densities [n_R, n_Z] of the cells at centres (R, Z) [n_R, n_Z]
    with temperatures T and volumes V, radial cell edges R_edges [n_R + 1]
    and column surface densities Sigma_g [n_R] (the mass per unit area of
    the cells of the column)."""
    R = np.asarray(R, dtype=np.float64)
    n_R, n_Z = R.shape
    rho = np.zeros((n_R, n_Z))
    for i in range(n_R):
        cs2 = [k_B * float(T[i][j]) / (mu * m_H) for j in range(n_Z)]
        r = [math.sqrt(float(R[i][j]) ** 2 + float(Z[i][j]) ** 2) for j in range(n_Z)]
        P = [1.0]                                   # P_{i,j} / P_{i,0}
        for j in range(1, n_Z):
            inv_cs2 = 0.5 * (1.0 / cs2[j] + 1.0 / cs2[j - 1])
            ratio = math.exp(GM * inv_cs2 * (1.0 / r[j] - 1.0 / r[j - 1]))
            P.append(P[j - 1] * ratio)
        omega = [P[j] / cs2[j] for j in range(n_Z)]
        RdR = 0.5 * (float(R_edges[i + 1]) ** 2 - float(R_edges[i]) ** 2)
        total = 0.0
        for j in range(n_Z):
            total += omega[j] * float(V[i][j])
        norm = float(Sigma_g[i]) * RdR / total
        for j in range(n_Z):
            rho[i, j] = norm * omega[j]
    return rho
