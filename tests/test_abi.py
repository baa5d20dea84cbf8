"""The C-ABI library loads, exports every function include/*.h declares, and
rejects bad arguments on the host before touching a device (no GPU needed)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2402_18471_b300 import coag, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(cudisc_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = coag.lib()
    names = declared_functions()
    assert "cudisc_coag_init" in names and "cudisc_coag_step" in names
    for n in names:
        assert hasattr(L, n), f"{n} is declared in include/ but not exported"


def test_version_string():
    assert "sm_103a" in coag.cudisc_coag_version()


def _params(disc, **over):
    p = coag.cudisc_coag_params()
    p.n_cells, p.n_bins = disc.n_cells, disc.n_bins
    keep = [np.ascontiguousarray(disc.m), np.ascontiguousarray(disc.me)]
    p.mass_centres, p.mass_edges = keep[0].ctypes.data, keep[1].ctypes.data
    # any non-NULL value passes the host checks; validation fails first
    for k in ("rho_gas", "T", "alpha", "R", "Z"):
        setattr(p, k, 16)
    s = disc.scalars()
    for k in ("v_frag", "eta_frag", "chi_im", "rho_m", "mu", "Mstar", "k_B", "m_H", "G",
              "sigma_H2", "kernel_const", "rtol", "atol_rel"):
        setattr(p, k, float(s[k]))
    p.max_substeps = 1000
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("field,value,code", [
    ("n_cells", 0, coag.EINVAL),
    ("n_bins", 1, coag.EINVAL),
    ("n_bins", 200, coag.ENOTSUP),
    ("rtol", 0.0, coag.EINVAL),
    ("max_substeps", 0, coag.EINVAL),
    ("precision", 7, coag.EINVAL),
    ("kernel_mode", 5, coag.EINVAL),
    ("rho_gas", None, coag.EINVAL),
    ("v_frag", -1.0, coag.EINVAL),
    ("mixed_cluster", 3, coag.EINVAL),
    ("mixed_cluster", 16, coag.EINVAL),
    ("max_sms", -1, coag.EINVAL),
    ("mixed_tile_stages", 9, coag.EINVAL),
    ("mixed_tile_stages", -1, coag.EINVAL),
    ("mixed_k_stages", 5, coag.EINVAL),
    ("cost_order", 2, coag.EINVAL),
])
def test_init_rejects_bad_arguments(field, value, code):
    d = synth.column_1x32()
    p, keep = _params(d, **{field: value})
    h = C.c_void_p()
    st = coag.lib().cudisc_coag_init(C.byref(p), C.byref(h))
    assert st == code
    assert h.value is None
    assert len(coag.lib().cudisc_coag_last_error(None)) > 0


def test_init_rejects_unbracketed_edges():
    d = synth.column_1x32()
    me = d.me.copy()
    me[10] = d.m[10] * 1.01         # edge above its own centre
    d.me = me
    p, keep = _params(d)
    h = C.c_void_p()
    assert coag.lib().cudisc_coag_init(C.byref(p), C.byref(h)) == coag.EINVAL
    assert b"bracket" in coag.lib().cudisc_coag_last_error(None)


def test_null_context_is_an_error_not_a_crash():
    L = coag.lib()
    assert L.cudisc_coag_build_kernel(None) == coag.EINVAL
    assert L.cudisc_coag_rhs(None, None, None) == coag.EINVAL
    assert L.cudisc_coag_step(None, None, 1.0, None, None) == coag.EINVAL
    assert L.cudisc_coag_vjp(None, None, 1.0, None, None, 0, None, None, None, None) == coag.EINVAL
    assert L.cudisc_coag_set_v_frag(None, 1.0) == coag.EINVAL
    assert L.cudisc_coag_set_adjoint_precision(None, 0) == coag.EINVAL
    t = coag.cudisc_timings()
    assert L.cudisc_coag_get_timings(None, C.byref(t)) == coag.EINVAL
    cl, gr = C.c_int(), C.c_int()
    assert L.cudisc_coag_mixed_cluster(None, C.byref(cl), C.byref(gr)) == coag.EINVAL
    assert L.cudisc_coag_step_async(None, None, 1.0, None) == coag.EINVAL
    assert L.cudisc_coag_step_wait(None, None) == coag.EINVAL
    h = C.c_void_p()
    assert L.cudisc_coag_init_batched(None, 0, C.byref(h)) == coag.EINVAL and h.value is None
    assert L.cudisc_coag_batch_ctx(None, 0, C.byref(h)) == coag.EINVAL
    assert L.cudisc_coag_batch_build_kernel(None) == coag.EINVAL
    assert L.cudisc_coag_batch_step(None, None, 1.0, None, None, None) == coag.EINVAL
    assert L.cudisc_coag_batch_step_async(None, None, 1.0, None, None) == coag.EINVAL
    assert L.cudisc_coag_batch_step_wait(None, None) == coag.EINVAL
    L.cudisc_coag_batch_destroy(None)
    L.cudisc_coag_destroy(None)
    assert L.cudisc_coag_build_kernel_async(None) == coag.EINVAL
    assert L.cudisc_coag_set_fault_injection(None, 0, 0) == coag.EINVAL
    n = C.c_size_t()
    assert L.cudisc_coag_scratch_bytes(None, C.byref(n)) == coag.EINVAL
    assert L.cudisc_coag_mixed_rings(None, C.byref(cl), C.byref(gr), C.byref(cl)) == coag.EINVAL
    assert L.cudisc_coag_step_host(None, None, None, 1.0, 0, None) == coag.EINVAL
    assert L.cudisc_dust_step(None, None, 1.0) == coag.EINVAL
    assert L.cudisc_dust_update_gas(None) == coag.EINVAL
    assert L.cudisc_dust_geometry(None, None, None, None) == coag.EINVAL
    L.cudisc_dust_destroy(None)


def test_transport_init_rejects_bad_arguments_before_any_allocation():
    L = coag.lib()
    Re = np.array([1.0, 2.0, 3.0])
    te = np.array([0.0, 0.1, 0.2])
    f = C.c_void_p(16)     # never dereferenced: validation fails first

    def params(**kw):
        p = coag.cudisc_dust_params()
        p.n_species, p.n_R, p.n_Z = 2, 2, 2
        p.R_e, p.th_e = Re.ctypes.data, te.ctypes.data
        p.rho_g = f.value
        for k, v in kw.items():
            if k == "bc":
                for i in range(4):
                    p.bc[i] = v[i]
            else:
                setattr(p, k, v)
        return p

    h = C.c_void_p()
    for kw, word in [(dict(n_species=0), b"n_species"), (dict(rho_g=None), b"rho_g"),
                     (dict(nu=f.value), b"Sc"), (dict(geometry=7), b"geometry"),
                     (dict(bc=(0, 0, 5, 0)), b"bc"), (dict(c_s=f.value), b"sources")]:
        p = params(**kw)
        assert L.cudisc_dust_init(C.byref(p), C.byref(h)) == coag.EINVAL and h.value is None
        assert word in L.cudisc_coag_last_error(None)
    bad = np.array([1.0, 0.5, 3.0])
    p = params()
    p.R_e = bad.ctypes.data
    assert L.cudisc_dust_init(C.byref(p), C.byref(h)) == coag.EINVAL
    assert b"R_e" in L.cudisc_coag_last_error(None)


def test_hse_rejects_bad_arguments_before_any_launch():
    L = coag.lib()
    fake = C.c_void_p(16)     # never dereferenced: validation fails first
    args = [fake] * 6
    assert L.cudisc_hse_rho_gas(0, 4, *args, 2.4, 1.67e-24, 1.38e-16, 1.3e26, fake, None) == coag.EINVAL
    assert L.cudisc_hse_rho_gas(3, 0, *args, 2.4, 1.67e-24, 1.38e-16, 1.3e26, fake, None) == coag.EINVAL
    assert L.cudisc_hse_rho_gas(3, 4, *args, 2.4, 1.67e-24, 1.38e-16, 1.3e26, None, None) == coag.EINVAL
    assert b"device arrays" in L.cudisc_coag_last_error(None)
    assert L.cudisc_hse_rho_gas(3, 4, *args, 2.4, 1.67e-24, 1.38e-16, -1.0, fake, None) == coag.EINVAL
    assert b"positive" in L.cudisc_coag_last_error(None)


def test_dust_calls_reject_bad_arguments_before_any_launch():
    L = coag.lib()
    f = C.c_void_p(16)     # never dereferenced: validation fails first
    assert L.cudisc_dust_source_update(0, 4, f, f, 1.0, f, f, f, f, f, f, 1.6, 1.0, None) == coag.EINVAL
    assert L.cudisc_dust_source_update(2, 4, None, f, 1.0, f, f, f, f, f, f, 1.6, 1.0, None) == coag.EINVAL
    assert L.cudisc_dust_source_update(2, 4, f, f, -1.0, f, f, f, f, f, f, 1.6, 1.0, None) == coag.EINVAL
    assert L.cudisc_dust_cfl_dt(2, 0, f, f, f, f, f, 0.4, 0.2, f, None) == coag.EINVAL
    assert L.cudisc_dust_cfl_dt(2, 4, f, f, f, f, f, 0.0, 0.2, f, None) == coag.EINVAL
    assert L.cudisc_dust_cfl_dt(2, 4, f, f, f, f, f, 0.4, 0.2, None, None) == coag.EINVAL
