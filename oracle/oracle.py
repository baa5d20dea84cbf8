"""ctypes wrapper of the FP64 CPU oracle (coag_oracle.c).

TEST INFRASTRUCTURE: imported only by tests, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The library path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coag_oracle.c")
_LIB = os.path.join(_HERE, "libcoag_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over cells)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class OracleParams(C.Structure):
    _fields_ = [
        ("n_cells", C.c_int), ("n_bins", C.c_int),
        ("m", C.c_void_p), ("me", C.c_void_p),
        ("rho_gas", C.c_void_p), ("T", C.c_void_p), ("alpha", C.c_void_p),
        ("R", C.c_void_p), ("Z", C.c_void_p), ("eta", C.c_void_p),
        ("v_dust", C.c_void_p),
        ("v_frag", C.c_double), ("eta_frag", C.c_double), ("chi_im", C.c_double),
        ("rho_m", C.c_double), ("mu", C.c_double), ("Mstar", C.c_double),
        ("k_B", C.c_double), ("m_H", C.c_double), ("G", C.c_double),
        ("sigma_H2", C.c_double),
        ("kernel_const", C.c_double),
        ("kernel_mode", C.c_int), ("frag_mode", C.c_int), ("split_mode", C.c_int),
        ("n_threads", C.c_int),
        ("rtol", C.c_double), ("atol_rel", C.c_double),
        ("max_substeps", C.c_long),
        ("vertical", C.c_int),
        ("kernel_perturb", C.c_double),
        ("perturb_seed", C.c_ulonglong),
        ("stage_noise", C.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER(OracleParams)
        d = C.c_void_p
        _lib.oracle_vrel2.restype = C.c_double
        _lib.oracle_vrel2.argtypes = [C.c_double, C.c_double, C.c_double]
        _lib.oracle_pfrag.restype = C.c_double
        _lib.oracle_pfrag.argtypes = [C.c_double, C.c_double]
        _lib.oracle_threads.restype = C.c_int
        _lib.oracle_cell_physics.argtypes = [P, C.c_int, d, d, d, d, d, d, d]
        _lib.oracle_kernel.argtypes = [P, d, d, d]
        _lib.oracle_pair_map.argtypes = [P, C.c_int, C.c_int, d, d]
        _lib.oracle_frag_table.argtypes = [P, d]
        _lib.oracle_rhs.argtypes = [P, d, d]
        _lib.oracle_rhs_bruteforce.argtypes = [P, d, d]
        _lib.oracle_step.argtypes = [P, d, C.c_double, d, d, d, d, d, C.c_long, d]
        _lib.oracle_step_replay.argtypes = [P, d, d, d, C.c_long]
        _lib.oracle_step_spans.argtypes = [P, d, d, d, d, d, d, d, C.c_long, d]
        _lib.oracle_bs3_scalar.argtypes = [C.c_double] * 6 + [C.c_int, C.c_long, d]
        _lib.oracle_vjp.argtypes = [P, d, d, d, C.c_long, d, d, d, d]
        for fn in ("oracle_cell_physics", "oracle_kernel", "oracle_pair_map",
                   "oracle_frag_table", "oracle_rhs", "oracle_rhs_bruteforce",
                   "oracle_step", "oracle_step_replay", "oracle_step_spans", "oracle_bs3_scalar", "oracle_vjp"):
            getattr(_lib, fn).restype = C.c_int
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Binds one synthetic Disc to the oracle (keeps the arrays alive)."""

    def __init__(self, disc, n_threads: int = 0, **over):
        self.disc = disc
        self._keep = {}
        s = disc.scalars()
        s.update(over)
        p = OracleParams()
        p.n_cells, p.n_bins = disc.n_cells, disc.n_bins
        for name in ("m", "me", "rho_gas", "T", "alpha", "R", "Z", "eta"):
            arr = _f64(getattr(disc, name))
            self._keep[name] = arr
            setattr(p, name, _ptr(arr))
        if disc.v_dust is not None:
            vd = _f64(disc.v_dust)
            self._keep["v_dust"] = vd
            p.v_dust = _ptr(vd)
        else:
            p.v_dust = None
        for k in ("v_frag", "eta_frag", "chi_im", "rho_m", "mu", "Mstar", "k_B", "m_H",
                  "G", "sigma_H2", "kernel_const", "rtol", "atol_rel"):
            setattr(p, k, float(s[k]))
        for k in ("kernel_mode", "frag_mode", "split_mode"):
            setattr(p, k, int(s[k]))
        p.max_substeps = int(s["max_substeps"])
        p.vertical = int(s.get("vertical", 0))
        # sensitivity runs only (not the method): K (1 + kernel_perturb u)
        # and, in replays, stage inputs (1 + stage_noise u), u uniform
        p.kernel_perturb = float(s.get("kernel_perturb", 0.0))
        p.perturb_seed = int(s.get("perturb_seed", 0))
        p.stage_noise = float(s.get("stage_noise", 0.0))
        p.n_threads = int(n_threads)
        self.p = p
        self.N = disc.n_bins
        self.n_cells = disc.n_cells

    # -- per-pair pieces -----------------------------------------------------
    def cell_physics(self, c):
        N = self.N
        a, St, vR, vp, vZ, h = (np.zeros(N) for _ in range(6))
        sc = np.zeros(3)
        lib().oracle_cell_physics(C.byref(self.p), c, _ptr(a), _ptr(St), _ptr(vR),
                                  _ptr(vp), _ptr(vZ), _ptr(h), _ptr(sc))
        return dict(a=a, St=St, vR=vR, vphi=vp, vZ=vZ, h=h, cs=sc[0], Re=sc[1], Vg2=sc[2])

    def kernel(self):
        N, nc = self.N, self.n_cells
        K = np.zeros((nc, N, N)); pf = np.zeros((nc, N, N)); dv = np.zeros((nc, N, N))
        lib().oracle_kernel(C.byref(self.p), _ptr(K), _ptr(pf), _ptr(dv))
        return K, pf, dv

    def pair_map(self, i, j):
        oi = np.zeros(5, dtype=np.int32); od = np.zeros(6)
        lib().oracle_pair_map(C.byref(self.p), i, j, _ptr(oi), _ptr(od))
        return oi, od

    def frag_table(self):
        t = np.zeros((self.N, self.N))
        lib().oracle_frag_table(C.byref(self.p), _ptr(t))
        return t

    # -- right-hand side and integration ------------------------------------
    def rhs(self, rho):
        rho = _f64(rho); out = np.zeros_like(rho)
        lib().oracle_rhs(C.byref(self.p), _ptr(rho), _ptr(out))
        return out

    def rhs_bruteforce(self, rho):
        rho = _f64(rho); out = np.zeros_like(rho)
        lib().oracle_rhs_bruteforce(C.byref(self.p), _ptr(rho), _ptr(out))
        return out

    def step(self, rho, t_span, dt=None, log_cap=0):
        """BS3 integration of every cell over t_span: one number for all
        cells, or an array of per-cell spans (cells with a span <= 0 are not
        touched)."""
        y = _f64(rho).copy()
        nc = self.n_cells
        dtv = np.zeros(nc) if dt is None else _f64(dt).copy()
        na = np.zeros(nc, dtype=np.int64); nr = np.zeros(nc, dtype=np.int64)
        stt = np.zeros(nc, dtype=np.int32)
        log = np.zeros((nc, max(log_cap, 1)))
        nl = np.zeros(nc, dtype=np.int64)
        if np.ndim(t_span):
            spans = _f64(t_span).reshape(-1)
            assert spans.size == nc
            rc = lib().oracle_step_spans(C.byref(self.p), _ptr(y), _ptr(spans), _ptr(dtv), _ptr(na),
                                         _ptr(nr), _ptr(stt), _ptr(log) if log_cap else None,
                                         int(log_cap), _ptr(nl))
        else:
            rc = lib().oracle_step(C.byref(self.p), _ptr(y), float(t_span), _ptr(dtv), _ptr(na),
                                   _ptr(nr), _ptr(stt), _ptr(log) if log_cap else None,
                                   int(log_cap), _ptr(nl))
        return dict(rho=y, dt=dtv, n_acc=na, n_rej=nr, status=stt, rc=rc,
                    log=log[:, :log_cap] if log_cap else None, n_log=nl)

    def subcycle(self, rho, pending, dt, dt_global, trigger=1.0, log_cap=0):
        """One global time step of a sub-cycled coagulation update (Sec. 6).

        The coagulation solver takes its own sub-steps; a cell is brought up
        to date once the global time elapsed since its last update (pending,
        plus this step's dt_global) has reached trigger x its last sub-step
        dt[c] (trigger 1 is the paper's default), or when it has no sub-step
        yet (dt[c] <= 0).  Such a cell is integrated over its whole pending
        time, which restarts at 0; the others only accumulate.  Returns the
        step() result (rho, dt, counts and logs after the update) with the
        spans used and the new pending times."""
        pending = _f64(pending).reshape(-1)
        dt = _f64(dt).reshape(-1)
        acc = pending + dt_global
        due = ~(dt > 0.0) | (acc >= trigger * dt)
        spans = np.where(due, acc, 0.0)
        res = self.step(rho, spans, dt, log_cap)
        res["spans"] = spans
        res["pending"] = np.where(due, 0.0, acc)
        return res

    def vjp(self, rho0, hs, n_h, w):
        """Gradient of sum(w * rho(T)) after replaying hs w.r.t. rho0, alpha, v_frag."""
        rho0 = _f64(rho0); hs = _f64(hs); w = _f64(w)
        n_h = np.ascontiguousarray(n_h, dtype=np.int64)
        g_rho0 = np.zeros_like(rho0); g_alpha = np.zeros(self.n_cells); g_vf = np.zeros(1)
        lib().oracle_vjp(C.byref(self.p), _ptr(rho0), _ptr(hs), _ptr(n_h), hs.shape[1], _ptr(w),
                         _ptr(g_rho0), _ptr(g_alpha), _ptr(g_vf))
        return g_rho0, g_alpha, float(g_vf[0])

    def replay(self, rho, hs, n_h):
        y = _f64(rho).copy()
        hs = _f64(hs)
        n_h = np.ascontiguousarray(n_h, dtype=np.int64)
        lib().oracle_step_replay(C.byref(self.p), _ptr(y), _ptr(hs), _ptr(n_h), hs.shape[1])
        return y


def replay_spread(disc, rho, hs, n_h, kernel_perturb=0.0, stage_noise=0.0, seeds=(1, 2, 3)):
    """Sensitivity of a replayed integration: the unperturbed replay y0 and,
    per element, the largest |y_s - y0| over replays whose kernel is
    perturbed by a relative kernel_perturb u per cell and pair, and/or whose
    stage inputs are perturbed by a relative stage_noise u at every stage
    (u uniform in [-1/2, 1/2), seed s).

    Once a cell settles into a coagulation-fragmentation balance, the
    explicit integrator at the paper's tolerance runs near its stability
    limit and changes of the right-hand side that vary from one evaluation
    to the next grow over thousands of steps; two correct implementations
    whose arithmetic differs at that level then differ by about this
    spread."""
    y0 = Oracle(disc).replay(rho, hs, n_h)
    spread = np.zeros_like(y0)
    for s in seeds:
        y = Oracle(disc, kernel_perturb=kernel_perturb, stage_noise=stage_noise,
                   perturb_seed=s).replay(rho, hs, n_h)
        spread = np.maximum(spread, np.abs(y - y0))
    return y0, spread


def vrel2(St1, St2, Re):
    return lib().oracle_vrel2(float(St1), float(St2), float(Re))


def pfrag(dv, vf):
    return lib().oracle_pfrag(float(dv), float(vf))


def bs3_scalar(lam, y0, t_span, h0, rtol=1e-6, atol=1e-12, fixed_steps=0):
    out = np.zeros(3)
    mode = 1 if fixed_steps else 0
    lib().oracle_bs3_scalar(float(lam), float(y0), float(t_span), float(h0), float(rtol),
                            float(atol), mode, int(fixed_steps), _ptr(out))
    return out


def threads() -> int:
    return lib().oracle_threads()
