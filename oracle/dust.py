"""dust.py -- plain FP64 CPU oracle of two pieces of the dust dynamics step of
Sec. 3.1 of Robinson, Booth & Owen, "Introducing cuDisc" (arXiv 2402.18471):
the source update of the full step and the CFL time step.

TEST INFRASTRUCTURE.  Only the tests and bench.py's CPU legs use it; it shares
no code with the CUDA library.

Conserved quantities per species s and cell c (Eq. quants):
  Q = (rho, rho v_R, rho v_phi R, rho v_Z).
Source update (the full step's items ii-iv, and vi-viii with the whole step):
  1. Q** = Q* + h S_exp(P^n), with the explicit sources (Eq. sources without
     drag or external forces) evaluated on the primitives P^n at the start of
     the step: 0, rho v_phi^2 / R - rho Omega^2 R, 0, -rho Omega^2 Z, with
     Omega^2 = G M_* / (R^2 + Z^2)^(3/2);
  2. Q** -> P**: v_R = Q_1 / rho, v_phi = Q_2 / (rho R), v_Z = Q_3 / rho;
  3. the drag update of the primitive velocities, implicit and exact for its
     linear diagonal system: v <- v - h / (h + t_s) (v - v_g), with the
     Epstein stopping time t_s = rho_m a / (rho_g v_th), v_th = sqrt(8/pi) c_s
     (Eq. t_stop);
  4. back to conserved quantities.
  h is half the step for the half-step update, the whole step for the full one.
CFL time step (Eqs. dtCFL, dt_adv, dt_diff):
  dt = min(C_adv min |dR / v_R|, |dZ / v_Z|;  C_diff min dR^2 Sc / nu, dZ^2 Sc / nu)
  over cells and species, with C_adv = 0.4 and C_diff = 0.2 by default.
Readings: Sec. 3.1 writes the velocities of the drag update as primitives and
the sources with v_phi; the angular-momentum source is drag alone (no explicit
term).  A zero velocity component imposes no advective limit.
Parity: pinned (tests/test_oracle_dust.py: Keplerian equilibrium, angular
momentum, the drag update's limits and backward-Euler form, CFL by brute force
on the definition).
"""
from __future__ import annotations

import math

import numpy as np


def source_update(Q, Pn, h, R, Z, rho_g, c_s, v_g, a, rho_m, GM):
    """Q, Pn: [4, n_species, n_cells] (conserved after transport; primitives
    rho, v_R, v_phi, v_Z at the start of the step).  R, Z, rho_g, c_s:
    [n_cells]; v_g: [3, n_cells]; a: [n_species] grain radii.  Returns the
    updated conserved quantities."""
    Q = np.array(Q, dtype=np.float64)
    Pn = np.asarray(Pn, dtype=np.float64)
    n_s, n_c = Q.shape[1], Q.shape[2]
    out = np.zeros_like(Q)
    for s in range(n_s):
        for c in range(n_c):
            Rc, Zc = float(R[c]), float(Z[c])
            Om2 = GM / (Rc * Rc + Zc * Zc) ** 1.5
            rho_n, vR_n, vphi_n, vZ_n = (float(Pn[f, s, c]) for f in range(4))
            # 1. explicit sources on the start-of-step primitives
            q0 = Q[0, s, c]
            q1 = Q[1, s, c] + h * (rho_n * vphi_n * vphi_n / Rc - rho_n * Om2 * Rc)
            q2 = Q[2, s, c]
            q3 = Q[3, s, c] + h * (-rho_n * Om2 * Zc)
            # 2. primitives
            vR, vphi, vZ = q1 / q0, q2 / (q0 * Rc), q3 / q0
            # 3. implicit drag
            vth = math.sqrt(8.0 / math.pi) * float(c_s[c])
            ts = rho_m * float(a[s]) / (float(rho_g[c]) * vth)
            f = h / (h + ts)
            vR = vR - f * (vR - float(v_g[0, c]))
            vphi = vphi - f * (vphi - float(v_g[1, c]))
            vZ = vZ - f * (vZ - float(v_g[2, c]))
            # 4. conserved
            out[0, s, c] = q0
            out[1, s, c] = q0 * vR
            out[2, s, c] = q0 * vphi * Rc
            out[3, s, c] = q0 * vZ
    return out


def cfl_dt(v_R, v_Z, dR, dZ, nu, Sc, C_adv=0.4, C_diff=0.2):
    """v_R, v_Z: [n_species, n_cells]; dR, dZ, nu: [n_cells]; Sc: [n_species]."""
    n_s, n_c = np.shape(v_R)
    adv = math.inf
    dif = math.inf
    for s in range(n_s):
        for c in range(n_c):
            for d, v in ((dR[c], v_R[s][c]), (dZ[c], v_Z[s][c])):
                if v != 0.0:
                    adv = min(adv, abs(d / v))
                dif = min(dif, abs(d * d / (nu[c] / Sc[s])))
    return min(C_adv * adv, C_diff * dif)
