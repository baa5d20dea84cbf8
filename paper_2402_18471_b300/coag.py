"""Thin Python binding of the C ABI in include/cudisc_coag.h.

Argument marshalling only: every step of the coagulation update runs in the
CUDA library libcudisc_coag.so.  PyTorch provides device memory and streams.
If the library cannot be loaded the binding raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

OK, EINVAL, ENOMEM, ECUDA, EMAXSTEPS, ENONFINITE, ENOTSUP, EDTMIN = range(8)
FP64, MIXED_TF32 = 0, 1
PRECISIONS = {"fp64": FP64, "mixed": MIXED_TF32, "mixed_tf32": MIXED_TF32}


class CoagError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cudisc status {status}: {msg}")
        self.status = status


class cudisc_coag_params(C.Structure):
    _fields_ = [
        ("n_cells", C.c_int), ("n_bins", C.c_int),
        ("mass_centres", C.c_void_p), ("mass_edges", C.c_void_p),
        ("rho_gas", C.c_void_p), ("T", C.c_void_p), ("alpha", C.c_void_p),
        ("R", C.c_void_p), ("Z", C.c_void_p), ("eta", C.c_void_p), ("v_dust", C.c_void_p),
        ("v_frag", C.c_double), ("eta_frag", C.c_double), ("chi_im", C.c_double),
        ("rho_m", C.c_double), ("mu", C.c_double), ("Mstar", C.c_double),
        ("k_B", C.c_double), ("m_H", C.c_double), ("G", C.c_double), ("sigma_H2", C.c_double),
        ("kernel_const", C.c_double),
        ("kernel_mode", C.c_int), ("frag_mode", C.c_int), ("split_mode", C.c_int),
        ("precision", C.c_int),
        ("rtol", C.c_double), ("atol_rel", C.c_double),
        ("max_substeps", C.c_longlong),
        ("stream", C.c_void_p),
        ("mixed_cluster", C.c_int),
        ("max_sms", C.c_int),
        ("vertical", C.c_int), ("mixed_pair", C.c_int),
        ("mixed_tile_stages", C.c_int), ("mixed_k_stages", C.c_int), ("cost_order", C.c_int),
    ]


class cudisc_dust_params(C.Structure):
    _fields_ = [
        ("n_species", C.c_int), ("n_R", C.c_int), ("n_Z", C.c_int),
        ("R_e", C.c_void_p), ("th_e", C.c_void_p), ("R_c", C.c_void_p), ("th_c", C.c_void_p),
        ("geometry", C.c_int), ("bc", C.c_int * 4), ("floor", C.c_double),
        ("rho_g", C.c_void_p), ("nu", C.c_void_p), ("Sc", C.c_void_p),
        ("c_s", C.c_void_p), ("v_g", C.c_void_p), ("a", C.c_void_p),
        ("rho_m", C.c_double), ("GM", C.c_double), ("stream", C.c_void_p),
    ]


class cudisc_timings(C.Structure):
    _fields_ = [("prep_ms", C.c_double), ("kbuild_ms", C.c_double),
                ("step_ms", C.c_double), ("vjp_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cudisc_step_stats(C.Structure):
    _fields_ = [
        ("accepted", C.c_longlong), ("rejected", C.c_longlong),
        ("max_accepted", C.c_longlong), ("n_failed", C.c_int), ("worst_status", C.c_int),
        ("mass_err_max", C.c_double), ("elapsed_ms", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libcudisc_coag.so (building it with nvcc when missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libcudisc_coag.so is missing and could not be built")
        L = C.CDLL(path)
        v, d = C.c_void_p, C.c_double
        L.cudisc_coag_init.argtypes = [C.POINTER(cudisc_coag_params), C.POINTER(v)]
        L.cudisc_coag_build_kernel.argtypes = [v]
        L.cudisc_coag_build_kernel_async.argtypes = [v]
        L.cudisc_coag_get_kernel.argtypes = [v, v, v]
        L.cudisc_coag_rhs.argtypes = [v, v, v]
        L.cudisc_coag_step.argtypes = [v, v, d, v, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_step_async.argtypes = [v, v, d, v]
        L.cudisc_coag_step_wait.argtypes = [v, C.POINTER(cudisc_step_stats)]
        L.cudisc_hse_rho_gas.argtypes = [C.c_int, C.c_int, v, v, v, v, v, v, d, d, d, d, v, v]
        L.cudisc_dust_source_update.argtypes = [C.c_int, C.c_int, v, v, d, v, v, v, v, v, v, d, d, v]
        L.cudisc_dust_cfl_dt.argtypes = [C.c_int, C.c_int, v, v, v, v, v, d, d, v, v]
        L.cudisc_coag_step_spans.argtypes = [v, v, v, v, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_subcycle.argtypes = [v, v, d, d, v, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_subcycle_pending.argtypes = [v, v, C.c_int]
        L.cudisc_coag_init_batched.argtypes = [C.POINTER(cudisc_coag_params), C.c_int, C.POINTER(v)]
        L.cudisc_coag_batch_ctx.argtypes = [v, C.c_int, C.POINTER(v)]
        L.cudisc_coag_batch_build_kernel.argtypes = [v]
        L.cudisc_coag_batch_step.argtypes = [v, C.POINTER(v), d, C.POINTER(v), v, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_batch_destroy.argtypes = [v]
        L.cudisc_coag_batch_destroy.restype = None
        L.cudisc_coag_set_records.argtypes = [v, v, C.c_longlong, v, v]
        L.cudisc_coag_replay.argtypes = [v, v, v, v, C.c_longlong]
        L.cudisc_coag_step_static_scratch.argtypes = [v, v, d, v, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_step_host.argtypes = [v, v, v, d, C.c_int, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_get_timings.argtypes = [v, C.POINTER(cudisc_timings)]
        L.cudisc_coag_mixed_cluster.argtypes = [v, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.cudisc_coag_scratch_bytes.argtypes = [v, C.POINTER(C.c_size_t)]
        L.cudisc_coag_mixed_pair.argtypes = [v, C.POINTER(C.c_int)]
        L.cudisc_coag_mixed_rings.argtypes = [v, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.cudisc_coag_set_fault_injection.argtypes = [v, C.c_longlong, C.c_int]
        L.cudisc_partition.argtypes = [C.c_int, v, C.c_int, v]
        L.cudisc_dust_init.argtypes = [C.POINTER(cudisc_dust_params), C.POINTER(v)]
        L.cudisc_dust_update_gas.argtypes = [v]
        L.cudisc_dust_step.argtypes = [v, v, d]
        L.cudisc_dust_geometry.argtypes = [v, v, v, v]
        L.cudisc_dust_destroy.argtypes = [v]
        L.cudisc_dust_destroy.restype = None
        L.cudisc_coag_set_v_frag.argtypes = [v, d]
        L.cudisc_coag_set_adjoint_precision.argtypes = [v, C.c_int]
        L.cudisc_coag_batch_step_async.argtypes = [v, C.POINTER(v), d, C.POINTER(v), v]
        L.cudisc_coag_batch_step_wait.argtypes = [v, C.POINTER(cudisc_step_stats)]
        L.cudisc_coag_vjp.argtypes = [v, v, d, v, v, C.c_longlong, v, v, v, v]
        L.cudisc_coag_destroy.argtypes = [v]
        L.cudisc_coag_destroy.restype = None
        L.cudisc_coag_last_error.argtypes = [v]
        L.cudisc_coag_last_error.restype = C.c_char_p
        L.cudisc_coag_version.restype = C.c_char_p
        for fn in ("cudisc_coag_init", "cudisc_coag_build_kernel", "cudisc_coag_build_kernel_async", "cudisc_coag_get_kernel",
                   "cudisc_coag_rhs", "cudisc_coag_step", "cudisc_coag_set_records",
                   "cudisc_coag_replay", "cudisc_coag_step_static_scratch", "cudisc_coag_step_host",
                   "cudisc_coag_get_timings", "cudisc_coag_set_v_frag", "cudisc_coag_set_adjoint_precision", "cudisc_coag_vjp",
                   "cudisc_coag_mixed_cluster", "cudisc_coag_scratch_bytes", "cudisc_coag_mixed_pair", "cudisc_coag_mixed_rings", "cudisc_coag_set_fault_injection", "cudisc_partition", "cudisc_dust_init", "cudisc_dust_update_gas",
                   "cudisc_dust_step", "cudisc_dust_geometry", "cudisc_coag_step_async", "cudisc_coag_step_wait",
                   "cudisc_coag_init_batched", "cudisc_coag_batch_ctx", "cudisc_coag_batch_build_kernel",
                   "cudisc_dust_source_update", "cudisc_dust_cfl_dt", "cudisc_hse_rho_gas", "cudisc_coag_batch_step", "cudisc_coag_step_spans", "cudisc_coag_subcycle",
                   "cudisc_coag_subcycle_pending", "cudisc_coag_batch_step_async", "cudisc_coag_batch_step_wait"):
            getattr(L, fn).restype = C.c_int
        _lib = L
    return _lib


def _check(st: int, ctx=None):
    if st != OK:
        msg = lib().cudisc_coag_last_error(ctx).decode()
        raise CoagError(st, msg)


# ---- the ABI calls, same names -------------------------------------------

def cudisc_coag_init(params: cudisc_coag_params):
    h = C.c_void_p()
    _check(lib().cudisc_coag_init(C.byref(params), C.byref(h)))
    return h


def cudisc_coag_build_kernel(ctx):
    _check(lib().cudisc_coag_build_kernel(ctx), ctx)


def cudisc_coag_build_kernel_async(ctx):
    _check(lib().cudisc_coag_build_kernel_async(ctx), ctx)


def cudisc_coag_get_kernel(ctx, K_ptr, KF_ptr):
    _check(lib().cudisc_coag_get_kernel(ctx, K_ptr, KF_ptr), ctx)


def cudisc_coag_rhs(ctx, rho_ptr, drho_ptr):
    _check(lib().cudisc_coag_rhs(ctx, rho_ptr, drho_ptr), ctx)


def cudisc_coag_step(ctx, rho_ptr, t_span, dt_ptr, check=True):
    s = cudisc_step_stats()
    st = lib().cudisc_coag_step(ctx, rho_ptr, float(t_span), dt_ptr, C.byref(s))
    if check:
        _check(st, ctx)
    return st, s


def cudisc_coag_step_host(ctx, rho_in_ptr, rho_out_ptr, t_span, rebuild=True, check=True):
    """cudisc_coag_step from and to host arrays (pointers to [n_cells][N]
    float64 host memory, pinned for DMA copies)."""
    s = cudisc_step_stats()
    st = lib().cudisc_coag_step_host(ctx, rho_in_ptr, rho_out_ptr, float(t_span), 1 if rebuild else 0, C.byref(s))
    if check:
        _check(st, ctx)
    return st, s


def cudisc_coag_step_async(ctx, rho_ptr, t_span, dt_ptr):
    """Issue one integration on the context's stream (graph-capturable)."""
    _check(lib().cudisc_coag_step_async(ctx, rho_ptr, float(t_span), dt_ptr), ctx)


def cudisc_coag_step_wait(ctx, check=True):
    s = cudisc_step_stats()
    st = lib().cudisc_coag_step_wait(ctx, C.byref(s))
    if check:
        _check(st, ctx)
    return st, s


def cudisc_coag_step_spans(ctx, rho_ptr, spans_ptr, dt_ptr, check=True):
    s = cudisc_step_stats()
    st = lib().cudisc_coag_step_spans(ctx, rho_ptr, spans_ptr, dt_ptr, C.byref(s))
    if check:
        _check(st, ctx)
    return st, s


def cudisc_coag_subcycle(ctx, rho_ptr, dt_global, trigger, dt_ptr, check=True):
    s = cudisc_step_stats()
    st = lib().cudisc_coag_subcycle(ctx, rho_ptr, float(dt_global), float(trigger), dt_ptr, C.byref(s))
    if check:
        _check(st, ctx)
    return st, s


def cudisc_coag_subcycle_pending(ctx, pending_ptr, reset):
    _check(lib().cudisc_coag_subcycle_pending(ctx, pending_ptr, int(bool(reset))), ctx)


def cudisc_hse_rho_gas(n_R, n_Z, R_ptr, Z_ptr, T_ptr, V_ptr, Re_ptr, Sig_ptr, mu, m_H, k_B, GM, rho_ptr,
                       stream=None):
    _check(lib().cudisc_hse_rho_gas(int(n_R), int(n_Z), R_ptr, Z_ptr, T_ptr, V_ptr, Re_ptr, Sig_ptr,
                                    float(mu), float(m_H), float(k_B), float(GM), rho_ptr, stream))


def hse_rho_gas(R, Z, T, V, R_edges, Sigma_g, mu, m_H, k_B, GM, out=None):
    """Hydrostatic-equilibrium gas density [n_R, n_Z] on the GPU (Sec. 3.5)
    from device FP64 tensors R, Z, T, V [n_R, n_Z], R_edges [n_R + 1] and
    Sigma_g [n_R], on torch's current stream; out (optional) receives it."""
    import torch
    ts = [t.contiguous() for t in (R, Z, T, V, R_edges, Sigma_g)]
    for t in ts:
        assert t.dtype == torch.float64 and t.is_cuda
    n_R, n_Z = ts[0].shape
    assert ts[4].numel() == n_R + 1 and ts[5].numel() == n_R
    assert all(t.shape == (n_R, n_Z) for t in ts[1:4])
    if out is None:
        out = torch.empty((n_R, n_Z), dtype=torch.float64, device=ts[0].device)
    cudisc_hse_rho_gas(n_R, n_Z, *(t.data_ptr() for t in ts), mu, m_H, k_B, GM, out.data_ptr(),
                       torch.cuda.current_stream(ts[0].device).cuda_stream)
    return out


def dust_source_update(Q, P_n, h, R, Z, rho_g, c_s, v_g, a, rho_m, GM):
    """The dust source update of Sec. 3.1 (sources, then implicit drag) on
    device FP64 tensors: Q (updated in place) and P_n [4, n_species, n_cells],
    R, Z, rho_g, c_s [n_cells], v_g [3, n_cells], a [n_species]; on torch's
    current stream."""
    import torch
    n_s, n_c = Q.shape[1], Q.shape[2]
    ts = [t.contiguous() for t in (P_n, R, Z, rho_g, c_s, v_g, a)]
    assert Q.is_contiguous() and Q.dtype == torch.float64
    Pn_, R_, Z_, rg_, cs_, vg_, a_ = (t.data_ptr() for t in ts)
    _check(lib().cudisc_dust_source_update(n_s, n_c, Q.data_ptr(), Pn_, float(h), R_, Z_, rg_, cs_, vg_, a_,
                                           float(rho_m), float(GM),
                                           torch.cuda.current_stream(Q.device).cuda_stream))
    return Q


def dust_cfl_dt(P, dR, dZ, nu, Sc, C_adv=0.4, C_diff=0.2, out=None):
    """The CFL time step of Sec. 3.1: a three-element device tensor whose
    element 0 is the step (1 and 2 hold the reduction's partial results)."""
    import torch
    n_s, n_c = P.shape[1], P.shape[2]
    ts = [t.contiguous() for t in (P, dR, dZ, nu, Sc)]
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=P.device)
    _check(lib().cudisc_dust_cfl_dt(n_s, n_c, *(t.data_ptr() for t in ts), float(C_adv), float(C_diff),
                                    out.data_ptr(), torch.cuda.current_stream(P.device).cuda_stream))
    return out


GEOM = {"cylindrical": 0, "cartesian": 1}
BC_OUTFLOW, BC_CLOSED, BC_ZERO = 0, 1, 2


class DustTransport:
    """The dust transport step (Sec. 3.1-3.2) on an (R, theta) grid through
    cudisc_dust_init / _step.  Fields are torch float64 CUDA tensors: gas
    rho_g, nu [n_R, n_Z]; Sc [n_species]; sources (c_s [n_R, n_Z], v_g
    [3, n_R, n_Z], a [n_species], rho_m, GM) or None; Q [4, n_species, n_R,
    n_Z] (rho, rho v_R, rho v_phi R, rho v_Z)."""

    def __init__(self, R_e, th_e, n_species, rho_g, nu=None, Sc=None, R_c=None, th_c=None,
                 geometry="cylindrical", bc=(BC_OUTFLOW, BC_OUTFLOW, BC_CLOSED, BC_OUTFLOW), floor=0.0,
                 sources=None, stream=None):
        import torch
        self.torch = torch
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
        self._h = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in
                   (("R_e", R_e), ("th_e", th_e), ("R_c", R_c), ("th_c", th_c)) if v is not None}
        self.n_R, self.n_Z, self.n_species = len(R_e) - 1, len(th_e) - 1, int(n_species)
        self._d = {"rho_g": dev(rho_g)}
        if nu is not None:
            self._d["nu"] = dev(nu)
            self._d["Sc"] = dev(Sc)
        if sources is not None:
            for k in ("c_s", "v_g", "a"):
                self._d[k] = dev(sources[k])
        p = cudisc_dust_params()
        p.n_species, p.n_R, p.n_Z = self.n_species, self.n_R, self.n_Z
        for k in ("R_e", "th_e", "R_c", "th_c"):
            setattr(p, k, self._h[k].ctypes.data if k in self._h else None)
        p.geometry = GEOM[geometry]
        for k in range(4):
            p.bc[k] = int(bc[k])
        p.floor = float(floor)
        for k in ("rho_g", "nu", "Sc", "c_s", "v_g", "a"):
            setattr(p, k, self._d[k].data_ptr() if k in self._d else None)
        p.rho_m = float(sources["rho_m"]) if sources is not None else 0.0
        p.GM = float(sources["GM"]) if sources is not None else 0.0
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p.stream = self.stream.cuda_stream
        h = C.c_void_p()
        _check(lib().cudisc_dust_init(C.byref(p), C.byref(h)))
        self.ctx = h

    def step(self, Q, dt: float):
        """One full step of Q (in place; [4, n_species, n_R, n_Z] float64 CUDA)."""
        assert Q.is_contiguous() and Q.dtype == self.torch.float64
        assert tuple(Q.shape) == (4, self.n_species, self.n_R, self.n_Z)
        _check(lib().cudisc_dust_step(self.ctx, Q.data_ptr(), float(dt)))
        return Q

    def gas(self, name: str):
        """The context's device copy of a gas field ("rho_g", "nu", "Sc",
        "c_s", "v_g", "a"); after changing rho_g, nu or Sc in place call
        update_gas()."""
        return self._d[name]

    def update_gas(self):
        _check(lib().cudisc_dust_update_gas(self.ctx))

    def geometry(self):
        t = self.torch
        V = t.empty((self.n_R, self.n_Z), dtype=t.float64, device="cuda")
        AR = t.empty((self.n_R + 1, self.n_Z), dtype=t.float64, device="cuda")
        AZ = t.empty((self.n_R, self.n_Z + 1), dtype=t.float64, device="cuda")
        _check(lib().cudisc_dust_geometry(self.ctx, V.data_ptr(), AR.data_ptr(), AZ.data_ptr()))
        return V, AR, AZ

    def close(self):
        if getattr(self, "ctx", None):
            lib().cudisc_dust_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cudisc_coag_init_batched(params_list):
    arr = (cudisc_coag_params * len(params_list))(*params_list)
    h = C.c_void_p()
    _check(lib().cudisc_coag_init_batched(arr, len(params_list), C.byref(h)))
    return h


def cudisc_coag_batch_ctx(batch, i):
    h = C.c_void_p()
    _check(lib().cudisc_coag_batch_ctx(batch, int(i), C.byref(h)))
    return h


def cudisc_coag_batch_build_kernel(batch):
    _check(lib().cudisc_coag_batch_build_kernel(batch))


def cudisc_coag_batch_step(batch, rho_ptrs, t_span, dt_ptrs, stream_ptr, check=True):
    n = len(rho_ptrs)
    rho = (C.c_void_p * n)(*rho_ptrs)
    dt = (C.c_void_p * n)(*dt_ptrs) if dt_ptrs is not None else None
    stats = (cudisc_step_stats * n)()
    st = lib().cudisc_coag_batch_step(batch, rho, float(t_span), dt, stream_ptr, stats)
    if check:
        _check(st)
    return st, [x.as_dict() for x in stats]


def cudisc_coag_batch_step_async(batch, rho_ptrs, t_span, dt_ptrs, stream_ptr):
    n = len(rho_ptrs)
    rho = (C.c_void_p * n)(*rho_ptrs)
    dt = (C.c_void_p * n)(*dt_ptrs) if dt_ptrs is not None else None
    _check(lib().cudisc_coag_batch_step_async(batch, rho, float(t_span), dt, stream_ptr))


def cudisc_coag_batch_step_wait(batch, n, check=True):
    stats = (cudisc_step_stats * n)()
    st = lib().cudisc_coag_batch_step_wait(batch, stats)
    if check:
        _check(st)
    return st, [x.as_dict() for x in stats]


def cudisc_coag_batch_destroy(batch):
    lib().cudisc_coag_batch_destroy(batch)


def cudisc_coag_step_static_scratch(ctx, rho_ptr, t_span, dt_ptr, check=True):
    """The integration of cudisc_coag_step, with the integrator's scratch in a
    fixed device array inside the library: allocates no device memory."""
    s = cudisc_step_stats()
    st = lib().cudisc_coag_step_static_scratch(ctx, rho_ptr, float(t_span), dt_ptr, C.byref(s))
    if check:
        _check(st, ctx)
    return st, s


def cudisc_coag_set_records(ctx, dt_ptr, cap, n_ptr, status_ptr):
    _check(lib().cudisc_coag_set_records(ctx, dt_ptr, int(cap), n_ptr, status_ptr), ctx)


def cudisc_coag_replay(ctx, rho_ptr, hs_ptr, n_ptr, stride):
    _check(lib().cudisc_coag_replay(ctx, rho_ptr, hs_ptr, n_ptr, int(stride)), ctx)


def cudisc_coag_set_v_frag(ctx, v_frag: float):
    _check(lib().cudisc_coag_set_v_frag(ctx, float(v_frag)), ctx)


ADJOINT_PRECISIONS = {"fp64": 0, "double_float": 1}   # cudisc_adjoint_precision


def cudisc_coag_set_adjoint_precision(ctx, precision):
    p = ADJOINT_PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().cudisc_coag_set_adjoint_precision(ctx, p), ctx)


def cudisc_coag_vjp(ctx, rho0_ptr, t_span, hs_ptr, n_ptr, stride, grad_rhoT_ptr, grad_rho0_ptr,
                    grad_alpha_ptr, grad_vfrag_ptr):
    _check(lib().cudisc_coag_vjp(ctx, rho0_ptr, float(t_span), hs_ptr, n_ptr, int(stride),
                                 grad_rhoT_ptr, grad_rho0_ptr, grad_alpha_ptr, grad_vfrag_ptr), ctx)


def cudisc_coag_get_timings(ctx) -> dict:
    t = cudisc_timings()
    _check(lib().cudisc_coag_get_timings(ctx, C.byref(t)), ctx)
    return t.as_dict()


def cudisc_coag_mixed_cluster(ctx) -> tuple:
    """(CTAs per slot group, groups) of the mixed kernel; (0, 0) for FP64."""
    cl, gr = C.c_int(), C.c_int()
    _check(lib().cudisc_coag_mixed_cluster(ctx, C.byref(cl), C.byref(gr)), ctx)
    return cl.value, gr.value


def cudisc_coag_set_fault_injection(ctx, wait_cycles: int, withhold: int):
    _check(lib().cudisc_coag_set_fault_injection(ctx, int(wait_cycles), int(withhold)), ctx)


def cudisc_coag_scratch_bytes(ctx) -> int:
    n = C.c_size_t()
    _check(lib().cudisc_coag_scratch_bytes(ctx, C.byref(n)), ctx)
    return int(n.value)


def cudisc_partition(cost, n_parts: int, n_items: int = None):
    """Contiguous ranges of items (cells or whole discs) for n_parts GPUs,
    balanced by cost (None: equal costs); returns bounds [n_parts + 1]."""
    if cost is None:
        n, cp = int(n_items), None
    else:
        c = np.ascontiguousarray(cost, dtype=np.float64)
        n, cp = c.size, c.ctypes.data
    b = np.zeros(int(n_parts) + 1, dtype=np.int32)
    _check(lib().cudisc_partition(n, cp, int(n_parts), b.ctypes.data))
    return b


def cudisc_coag_destroy(ctx):
    lib().cudisc_coag_destroy(ctx)


def cudisc_coag_version() -> str:
    return lib().cudisc_coag_version().decode()


# ---- convenience wrapper over one synthetic disc ---------------------------

class Coag:
    """A context bound to one disc.  Gas arrays are copied to the device once;
    dust states are torch float64 CUDA tensors of shape [n_cells, N]."""

    def __init__(self, disc, precision: str = "fp64", device: str = "cuda", stream=None,
                 use_v_dust: bool = True, **over):
        import torch
        self._setup(disc, precision, device, use_v_dust, over)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params.stream = self.stream.cuda_stream
        self.ctx = cudisc_coag_init(self.params)
        self._owned = True
        self._rec = None

    def _setup(self, disc, precision, device, use_v_dust, over):
        """The disc's gas arrays on the device and its cudisc_coag_params."""
        import torch
        self.torch = torch
        self.disc = disc
        self.device = torch.device(device)
        self.N = disc.n_bins
        self.n_cells = disc.n_cells
        self.Np = self.N * (self.N + 1) // 2
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        s = disc.scalars()
        s.update(over)
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device)
        self._keep = {k: dev(getattr(disc, k)) for k in ("rho_gas", "T", "alpha", "R", "Z", "eta")}
        if use_v_dust and disc.v_dust is not None:
            self._keep["v_dust"] = dev(disc.v_dust)
        self._m = np.ascontiguousarray(disc.m, dtype=np.float64)
        self._me = np.ascontiguousarray(disc.me, dtype=np.float64)
        p = cudisc_coag_params()
        p.n_cells, p.n_bins = self.n_cells, self.N
        p.mass_centres = self._m.ctypes.data
        p.mass_edges = self._me.ctypes.data
        for k in ("rho_gas", "T", "alpha", "R", "Z", "eta"):
            setattr(p, k, self._keep[k].data_ptr())
        p.v_dust = self._keep["v_dust"].data_ptr() if "v_dust" in self._keep else None
        for k in ("v_frag", "eta_frag", "chi_im", "rho_m", "mu", "Mstar", "k_B", "m_H", "G",
                  "sigma_H2", "kernel_const", "rtol", "atol_rel"):
            setattr(p, k, float(s[k]))
        for k in ("kernel_mode", "frag_mode", "split_mode"):
            setattr(p, k, int(s[k]))
        p.precision = self.precision
        p.max_substeps = int(s["max_substeps"])
        p.mixed_cluster = int(s.get("mixed_cluster", 0))
        p.max_sms = int(s.get("max_sms", 0))
        p.vertical = int(s.get("vertical", 0))
        p.mixed_pair = int(s.get("mixed_pair", 0))
        p.mixed_tile_stages = int(s.get("mixed_tile_stages", 0))
        p.mixed_k_stages = int(s.get("mixed_k_stages", 0))
        p.cost_order = int(s.get("cost_order", 0))
        self.params = p

    def close(self):
        if getattr(self, "ctx", None):
            if getattr(self, "_owned", True):
                cudisc_coag_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state(self, rho):
        return self.torch.as_tensor(np.ascontiguousarray(rho, dtype=np.float64), device=self.device)

    def build_kernel(self):
        cudisc_coag_build_kernel(self.ctx)

    def build_kernel_async(self):
        """Issue the kernel-table rebuild on the context's stream (graph-capturable)."""
        cudisc_coag_build_kernel_async(self.ctx)

    def scratch_bytes(self) -> int:
        return cudisc_coag_scratch_bytes(self.ctx)

    def timings(self) -> dict:
        return cudisc_coag_get_timings(self.ctx)

    def mixed_pair(self) -> int:
        """1 when the mixed kernel runs in CTA pairs sharing M = 256 MMAs."""
        v = C.c_int()
        _check(lib().cudisc_coag_mixed_pair(self.ctx, C.byref(v)), self.ctx)
        return v.value

    def mixed_cluster(self) -> tuple:
        """(CTAs per group of 64 slots, groups) of the mixed kernel."""
        return cudisc_coag_mixed_cluster(self.ctx)

    def mixed_rings(self) -> tuple:
        """(mapping-tile stages, K-table stages, per-slot state in shared
        memory 0/1) of the mixed kernel."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(lib().cudisc_coag_mixed_rings(self.ctx, C.byref(a), C.byref(b), C.byref(c)), self.ctx)
        return a.value, b.value, c.value

    def get_kernel(self):
        t = self.torch
        K = t.empty((self.n_cells, self.Np), dtype=t.float64, device=self.device)
        KF = t.empty_like(K)
        cudisc_coag_get_kernel(self.ctx, K.data_ptr(), KF.data_ptr())
        return K, KF

    def rhs(self, rho):
        rho = rho.contiguous()
        out = self.torch.empty_like(rho)
        cudisc_coag_rhs(self.ctx, rho.data_ptr(), out.data_ptr())
        return out

    def set_records(self, log_cap: int):
        t = self.torch
        if log_cap <= 0:
            cudisc_coag_set_records(self.ctx, None, 0, None, None)
            self._rec = None
            return None
        self._rec = dict(
            dt=t.zeros((self.n_cells, log_cap), dtype=t.float64, device=self.device),
            n=t.zeros(self.n_cells, dtype=t.int64, device=self.device),
            status=t.zeros(self.n_cells, dtype=t.int32, device=self.device))
        cudisc_coag_set_records(self.ctx, self._rec["dt"].data_ptr(), log_cap,
                                self._rec["n"].data_ptr(), self._rec["status"].data_ptr())
        return self._rec

    def step(self, rho, t_span, dt=None, check=True):
        """Integrate rho (in place) over t_span; returns the stats dict."""
        assert rho.is_contiguous() and rho.dtype == self.torch.float64
        st, s = cudisc_coag_step(self.ctx, rho.data_ptr(), t_span,
                                 dt.data_ptr() if dt is not None else None, check=check)
        d = s.as_dict()
        d["status"] = st
        return d

    def step_host(self, rho_in, rho_out, t_span, rebuild=True, check=True):
        """cudisc_coag_step_host: host float64 tensors or arrays [n_cells, N]
        in and out (may be the same; pin them for DMA copies), the kernel
        tables rebuilt first when rebuild; returns the stats dict."""
        def ptr(x):
            if hasattr(x, "data_ptr"):
                assert not x.is_cuda and x.is_contiguous() and x.dtype == self.torch.float64
                return x.data_ptr()
            assert x.flags["C_CONTIGUOUS"] and x.dtype == np.float64
            return x.ctypes.data
        st, s = cudisc_coag_step_host(self.ctx, ptr(rho_in), ptr(rho_out), t_span, rebuild, check=check)
        d = s.as_dict()
        d["status"] = st
        return d

    def step_async(self, rho, t_span, dt=None):
        """Issue the integration on the context's stream and return at once
        (graph-capturable); step_wait() then gives the stats dict."""
        assert rho.is_contiguous() and rho.dtype == self.torch.float64
        cudisc_coag_step_async(self.ctx, rho.data_ptr(), t_span, dt.data_ptr() if dt is not None else None)

    def step_wait(self, check=True):
        st, s = cudisc_coag_step_wait(self.ctx, check=check)
        d = s.as_dict()
        d["status"] = st
        return d

    def step_spans(self, rho, spans, dt=None, check=True):
        """Integrate cell c of rho (in place) over spans[c] (device FP64
        [n_cells]); cells with spans[c] <= 0 are left as they are."""
        assert rho.is_contiguous() and rho.dtype == self.torch.float64
        spans = spans.contiguous()
        assert spans.dtype == self.torch.float64 and spans.numel() == self.n_cells
        st, s = cudisc_coag_step_spans(self.ctx, rho.data_ptr(), spans.data_ptr(),
                                       dt.data_ptr() if dt is not None else None, check=check)
        d = s.as_dict()
        d["status"] = st
        return d

    def subcycle(self, rho, dt_global, dt=None, trigger=1.0, check=True):
        """One global step of dt_global: update the cells whose pending time
        has reached trigger x their last coagulation sub-step (Sec. 6)."""
        assert rho.is_contiguous() and rho.dtype == self.torch.float64
        st, s = cudisc_coag_subcycle(self.ctx, rho.data_ptr(), dt_global, trigger,
                                     dt.data_ptr() if dt is not None else None, check=check)
        d = s.as_dict()
        d["status"] = st
        return d

    def pending(self, reset=False):
        """The cells' pending (not yet integrated) global times."""
        out = self.torch.empty(self.n_cells, dtype=self.torch.float64, device=self.device)
        cudisc_coag_subcycle_pending(self.ctx, out.data_ptr(), reset)
        return out

    def replay(self, rho, hs, n_h):
        assert rho.is_contiguous()
        hs = hs.contiguous()
        n_h = n_h.contiguous().to(self.torch.int64)
        cudisc_coag_replay(self.ctx, rho.data_ptr(), hs.data_ptr(), n_h.data_ptr(), hs.shape[1])

    # -- parameters the adjoint differentiates ------------------------------
    def set_alpha(self, alpha):
        """Copy new per-cell alpha values into the array the context reads
        (call build_kernel afterwards)."""
        self._keep["alpha"].copy_(self.torch.as_tensor(alpha, dtype=self.torch.float64,
                                                       device=self.device).reshape(-1))

    def set_v_frag(self, v_frag: float):
        cudisc_coag_set_v_frag(self.ctx, float(v_frag))

    def set_adjoint_precision(self, precision):
        """Arithmetic of later vjp calls' per-pair work: "fp64" (default) or
        "double_float" (FP32 pairs on the FP32 pipes)."""
        cudisc_coag_set_adjoint_precision(self.ctx, precision)

    def vjp(self, rho0, grad_rhoT, hs=None, n_h=None, t_span=0.0):
        """Gradients of sum(grad_rhoT * rho(T)) with respect to rho0, the
        per-cell alpha and v_frag, for the given step sequence (hs, n_h) or,
        without one, for a fresh adaptive integration over t_span."""
        t = self.torch
        rho0 = rho0.contiguous()
        grad_rhoT = grad_rhoT.contiguous().to(t.float64)
        g0 = t.empty_like(rho0)
        ga = t.empty(self.n_cells, dtype=t.float64, device=self.device)
        gv = t.empty(1, dtype=t.float64, device=self.device)
        if hs is None:
            cudisc_coag_vjp(self.ctx, rho0.data_ptr(), t_span, None, None, 0, grad_rhoT.data_ptr(),
                            g0.data_ptr(), ga.data_ptr(), gv.data_ptr())
        else:
            hs = hs.contiguous()
            n_h = n_h.contiguous().to(t.int64)
            cudisc_coag_vjp(self.ctx, rho0.data_ptr(), 0.0, hs.data_ptr(), n_h.data_ptr(),
                            hs.shape[1], grad_rhoT.data_ptr(), g0.data_ptr(), ga.data_ptr(),
                            gv.data_ptr())
        return g0, ga, gv


def autotune_cluster(disc, t_probe=None, candidates=(1, 2, 4, 8), cache_path=None, device="cuda", **over):
    """Measured choice of the mixed kernel's cluster size (CTAs that split each
    pass of a slot group) for this problem's cell and bin counts.

    Each candidate runs one warm-up and one timed integration over t_probe
    (default: a tenth of disc.t_span) from disc.rho0; the best throughput in
    accepted cell-substeps per second wins.  Candidates whose buffers do not
    fit (the library falls back to a smaller size) are skipped.  With
    cache_path, results are kept in a JSON file keyed by (bins, cells,
    precision) and later calls read them instead of measuring.  Returns the
    cluster size, to pass as mixed_cluster."""
    import json
    import torch
    key = f"N{disc.n_bins}_cells{disc.n_cells}_mixed"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return int(cache[key]["best"])
    t = disc.t_span / 10.0 if t_probe is None else float(t_probe)
    rates = {}
    for P in candidates:
        g = Coag(disc, "mixed", device=device, mixed_cluster=P, **over)
        try:
            if g.mixed_cluster()[0] != P:
                continue
            for rep in range(2):
                y = g.state(disc.rho0)
                st = g.step(y, t)
            rates[P] = st["accepted"] / max(st["elapsed_ms"], 1e-9) * 1e3
        finally:
            g.close()
            torch.cuda.synchronize()
    if not rates:
        raise CoagError(ENOTSUP, "no cluster size fits this problem")
    best = max(rates, key=rates.get)
    if cache_path:
        cache[key] = {"best": int(best), "rates": {str(k): v for k, v in rates.items()}, "t_probe": t}
        d = os.path.dirname(os.path.abspath(cache_path))
        os.makedirs(d, exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return int(best)


RING_CANDIDATES = ((2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (4, 1))


def autotune_launch(disc, t_probe=None, clusters=(1, 2, 4, 8), pairs=(1, 2), rings=RING_CANDIDATES,
                    cache_path=None, device="cuda", **over):
    """Measured choice of the mixed kernel's launch layout for this problem:
    the cluster size (mixed_cluster: CTAs that split each pass of a slot
    group), the CTA-pair mode (mixed_pair = 2: two CTAs share each M = 256
    tensor-core MMA, each keeping half of every mapping tile; 1: single
    CTAs), then, for the best of those, the shared-memory ring depths
    (mixed_tile_stages, mixed_k_stages; (0, 0) = the library's own choice,
    which puts the per-slot state in shared memory first).  Every layout
    that fits gets one warm-up and one timed integration over t_probe
    (default: a tenth of disc.t_span) from disc.rho0; the best accepted
    cell-substeps per second wins.  With cache_path the results are kept in
    a JSON file keyed by (bins, cells, precision) and later calls read them
    instead of measuring.  Returns {"mixed_cluster": P, "mixed_pair": 1 or
    2, "mixed_tile_stages": SB, "mixed_k_stages": KS}, to pass to Coag."""
    import json
    import torch
    key = f"N{disc.n_bins}_cells{disc.n_cells}_mixed_launch"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key]["best"])
    t = disc.t_span / 10.0 if t_probe is None else float(t_probe)

    def probe(P, pair, sb, ks):
        try:
            g = Coag(disc, "mixed", device=device, mixed_cluster=P, mixed_pair=pair, mixed_tile_stages=sb,
                     mixed_k_stages=ks, **over)
        except CoagError as e:
            if e.status == EINVAL and (sb or ks):
                return None                    # these rings do not fit
            raise
        try:
            if g.mixed_cluster()[0] != P or g.mixed_pair() != (1 if pair == 2 else 0):
                return None                    # the library fell back: this layout does not fit
            if (sb or ks) and g.mixed_rings()[:2] != (sb, ks):
                return None
            for rep in range(2):
                y = g.state(disc.rho0)
                st = g.step(y, t)
            return st["accepted"] / max(st["elapsed_ms"], 1e-9) * 1e3
        finally:
            g.close()
            torch.cuda.synchronize()

    rates = {}
    for pair in pairs:
        for P in clusters:
            r = probe(P, pair, 0, 0)
            if r is not None:
                rates[(P, pair, 0, 0)] = r
    if not rates:
        raise CoagError(ENOTSUP, "no launch layout fits this problem")
    P, pair, _, _ = max(rates, key=rates.get)
    for sb, ks in rings:
        r = probe(P, pair, sb, ks)
        if r is not None:
            rates[(P, pair, sb, ks)] = r
    P, pair, sb, ks = max(rates, key=rates.get)
    best = {"mixed_cluster": int(P), "mixed_pair": int(pair), "mixed_tile_stages": int(sb),
            "mixed_k_stages": int(ks)}
    if cache_path:
        cache[key] = {"best": best, "rates": {f"P{k[0]}_pair{k[1]}_sb{k[2]}_ks{k[3]}": v for k, v in rates.items()},
                      "t_probe": t}
        d = os.path.dirname(os.path.abspath(cache_path))
        os.makedirs(d, exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best


class Batch:
    """Several discs integrated side by side through the batched interface:
    one context per disc (disc(i) gives a Coag view of it), SMs shared out in
    proportion to n_cells x n_bins^2."""

    def __init__(self, discs, precision: str = "mixed", device: str = "cuda", use_v_dust: bool = True,
                 **over):
        import torch
        self.torch = torch
        self.discs = list(discs)
        self._views = []
        for d in self.discs:
            v = Coag.__new__(Coag)
            v._setup(d, precision, device, use_v_dust, dict(over))
            v._owned = False
            v._rec = None
            self._views.append(v)
        self.handle = cudisc_coag_init_batched([v.params for v in self._views])
        for i, v in enumerate(self._views):
            v.ctx = cudisc_coag_batch_ctx(self.handle, i)
            v.stream = None

    def disc(self, i) -> "Coag":
        return self._views[i]

    def __len__(self):
        return len(self._views)

    def build_kernel(self):
        cudisc_coag_batch_build_kernel(self.handle)

    def step(self, rhos, t_span, dts=None, check=True):
        """Integrate every disc's state (in place) over t_span; per-disc stats."""
        stream = self.torch.cuda.current_stream().cuda_stream
        st, stats = cudisc_coag_batch_step(self.handle, [r.data_ptr() for r in rhos], t_span,
                                           [d.data_ptr() if d is not None else None for d in dts]
                                           if dts is not None else None, stream, check=check)
        for s in stats:
            s["status"] = s["worst_status"]
        return stats

    def step_async(self, rhos, t_span, dts=None):
        """Issue every disc's integration, forked from and joined back to
        torch's current stream, without synchronising (graph-capturable once
        a synchronous step() has run)."""
        stream = self.torch.cuda.current_stream().cuda_stream
        cudisc_coag_batch_step_async(self.handle, [r.data_ptr() for r in rhos], t_span,
                                     [d.data_ptr() if d is not None else None for d in dts]
                                     if dts is not None else None, stream)

    def step_wait(self, check=True):
        """Per-disc stats of the last issued batch step."""
        st, stats = cudisc_coag_batch_step_wait(self.handle, len(self._views), check=check)
        for s in stats:
            s["status"] = s["worst_status"]
        return stats

    def close(self):
        if getattr(self, "handle", None):
            for v in self._views:
                v.ctx = None
            cudisc_coag_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _coag_step_function():
    import torch

    class CoagStep(torch.autograd.Function):
        """rho(T) = step(rho0; alpha, v_frag) as a differentiable function.

        forward: sets alpha and v_frag on the context, rebuilds K and runs the
        adaptive integration over t_span with step records; backward: the
        library's adjoint over the recorded step sequence (the step sizes are
        held fixed, as in the discrete adjoint)."""

        @staticmethod
        def forward(ctx, rho0, alpha, v_frag, coag, t_span, log_cap):
            coag.set_alpha(alpha.detach())
            coag.set_v_frag(float(v_frag))
            coag.build_kernel()
            rec = coag.set_records(log_cap)
            y = rho0.detach().to(torch.float64).contiguous().clone()
            st = coag.step(y, t_span)
            coag.set_records(0)
            if int(rec["n"].max()) > log_cap:
                raise CoagError(ENOTSUP, f"more than log_cap={log_cap} accepted substeps in a cell")
            ctx.save_for_backward(rho0.detach(), alpha.detach())
            ctx.coag, ctx.v_frag = coag, float(v_frag)
            ctx.vf_shape = v_frag.shape if torch.is_tensor(v_frag) else None
            ctx.hs, ctx.n_h = rec["dt"], rec["n"]
            ctx.stats = st
            return y

        @staticmethod
        def backward(ctx, g):
            rho0, alpha = ctx.saved_tensors
            coag = ctx.coag
            coag.set_alpha(alpha)
            coag.set_v_frag(ctx.v_frag)
            coag.build_kernel()
            g0, ga, gv = coag.vjp(rho0.to(torch.float64), g, ctx.hs, ctx.n_h)
            g_vf = gv.reshape(ctx.vf_shape) if ctx.vf_shape is not None else None
            return g0.to(rho0.dtype), ga.reshape(alpha.shape).to(alpha.dtype), g_vf, None, None, None

    return CoagStep


_CoagStep = None


def coag_step(rho0, alpha, v_frag, coag: "Coag", t_span: float, log_cap: int = 4096):
    """Differentiable coagulation step: rho(T) from rho0 [n_cells, N] (CUDA
    float64), alpha [n_cells] and a scalar v_frag tensor; gradients flow to
    all three through cudisc_coag_vjp."""
    global _CoagStep
    if _CoagStep is None:
        _CoagStep = _coag_step_function()
    return _CoagStep.apply(rho0, alpha, v_frag, coag, t_span, log_cap)
