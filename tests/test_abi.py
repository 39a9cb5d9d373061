"""The C-ABI library builds, loads, exports every symbol include/cl_lattice.h
declares, and validates arguments on the host (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2006_15122_gb300 as cl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "cl_lattice.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^(?:cl_status|int32_t|int64_t|const char\s*\*)\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declarations_match_binding():
    assert _declared_functions() == sorted(cl.SYMBOLS)


def test_library_exports_every_declared_symbol():
    lib = cl.load()
    out = subprocess.run(["nm", "-D", "--defined-only", cl.library_path()], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    for name in _declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_header_compiles_as_c():
    r = subprocess.run(["gcc", "-fsyntax-only", "-Wall", "-Werror", "-x", "c", os.path.join(ROOT, "include", "cl_lattice.h")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_status_strings():
    lib = cl.load()
    for s in range(9):
        assert lib.cl_status_str(s)
    assert lib.cl_last_error(None)


def _init(model, grid, init):
    lib = cl.load()
    h = C.c_void_p()
    st = lib.lattice_init(C.byref(model), C.byref(grid), C.byref(init), None, C.byref(h))
    return st, h


@pytest.mark.parametrize("N", [4, 12, 4096])
def test_init_rejects_bad_lattice_size(N):
    st, h = _init(cl.make_model(), cl.make_grid(N, 0.5, 0.01), cl.make_init())
    assert st == cl.CL_ERR_ARG and not h.value
    assert b"N must be" in cl.load().cl_last_error(None)


def test_init_rejects_unstable_time_step():
    """omega_max dt above the leapfrog/VV2 bound 2 (VV4: 1.5734) is refused before any device work."""
    m = cl.make_model(n_fields=2, pexp=2, q=4e5, omega_over_fstar=5e-6, fstar_over_mp=1.4)
    st, h = _init(m, cl.make_grid(64, 0.1, 0.005, "vv4"), cl.make_init(phi0=(1.0, 0.0)))
    assert st == cl.CL_ERR_UNSTABLE_DT and not h.value
    assert b"stability bound" in cl.load().cl_last_error(None)


@pytest.mark.parametrize("bad", ["integrator", "pexp", "fields", "kir", "u1_charge", "u1_integrator",
                                 "gauge_potential", "gauge_pexp", "su2_fields", "su2_u1_charge", "noncompact_su2",
                                 "u1_too_many_sites"])
def test_init_rejects_bad_arguments(bad):
    m = cl.make_model(n_fields=1, pexp=2)
    g = cl.make_grid(16, 0.5, 0.01)
    if bad == "integrator":
        g.integrator = 42
    if bad == "pexp":
        m.pexp = 3
    if bad == "fields":
        m.n_fields = 3
    if bad == "kir":
        g.kIR = -1.0
    if bad == "u1_charge":
        m.kind = cl.CL_MODEL_U1
        m.gauge_e = 0.0
        g.integrator = cl.CL_INT_VV4
    if bad == "u1_integrator":
        m.kind = cl.CL_MODEL_U1
        m.gauge_e = 1.0
        g.integrator = 6
    if bad in ("gauge_potential", "gauge_pexp"):
        m.kind = cl.CL_MODEL_SU2
        m.gauge_e = 1.0
        m.potential = 2 if bad == "gauge_potential" else cl.CL_POT_MONOMIAL
        m.pexp = 3
    if bad in ("su2_fields", "su2_u1_charge"):
        m.kind = cl.CL_MODEL_SU2
        m.gauge_e = 1.0
        m.n_fields = 3 if bad == "su2_fields" else 1
        m.gauge_e_u1 = -1.0 if bad == "su2_u1_charge" else 0.0
    if bad == "u1_too_many_sites":  # 32-bit site indices of the U(1) pass
        m.kind = cl.CL_MODEL_U1
        m.gauge_e = 1.0
        g.N = 1632
    if bad == "noncompact_su2":  # the non-compact form exists for U(1) only
        m.kind = cl.CL_MODEL_SU2
        m.gauge_e = 1.0
        m.noncompact = 1
    st, h = _init(m, g, cl.make_init())
    assert st == cl.CL_ERR_ARG and not h.value


def test_null_arguments_are_rejected():
    lib = cl.load()
    assert lib.lattice_evolve(None, 1) == cl.CL_ERR_ARG
    assert lib.lattice_measure_means(None, None) == cl.CL_ERR_ARG
    assert lib.lattice_destroy(None) == cl.CL_OK


@pytest.mark.parametrize("dims", [(0, 34, 256, 3), (2, 0, 256, 3), (2, 34, 0, 3), (2, 34, 256, 0), (2, 34, 5000, 3),
                                  (2, 34, 256, 17)])
def test_surrogate_create_rejects_bad_sizes(dims):
    lib = cl.load()
    h = C.c_void_p()
    assert lib.surrogate_create(*dims, 0, None, C.byref(h)) == cl.CL_ERR_ARG and not h.value
    assert b"surrogate_create" in lib.cl_last_error(None)


def test_surrogate_null_arguments_are_rejected():
    lib = cl.load()
    assert lib.surrogate_create(2, 34, 256, 3, 0, None, None) == cl.CL_ERR_ARG
    assert lib.surrogate_param_count(None) == 0
    assert lib.surrogate_train(None, None, None, 1, None, None) == cl.CL_ERR_ARG
    assert lib.surrogate_predict(None, None, 1, None) == cl.CL_ERR_ARG
    assert lib.surrogate_loss_grad(None, None, None, 1, None, None) == cl.CL_ERR_ARG
    assert lib.surrogate_destroy(None) == cl.CL_OK


def test_noalloc_binding_rejects_host_tensors_and_wrong_dtypes():
    """energies_noalloc refuses, before any CUDA call, buffers that are not
    contiguous CUDA float64 tensors (the C side would read them as device memory)."""
    torch = pytest.importorskip("torch")
    model = cl.make_model(n_fields=1)
    t = torch.zeros(64, dtype=torch.float64)
    with pytest.raises(ValueError):
        cl.energies_noalloc(model, 4, 0.5, 1.0, t, t, torch.zeros(10, dtype=torch.float64))
    with pytest.raises(ValueError):
        cl.energies_noalloc(model, 4, 0.5, 1.0, t.float(), t.float(), t.float())


def test_noalloc_rejects_bad_arguments_on_the_host():
    lib = cl.load()
    m = cl.make_model(n_fields=3)
    assert lib.lattice_energies_noalloc(C.byref(m), 8, 0.5, 1.0, None, None, None, None) == cl.CL_ERR_ARG
    assert b"non-NULL" in lib.cl_last_error(None)
    dummy = C.c_void_p(16)  # never dereferenced: the model is rejected first
    assert lib.lattice_energies_noalloc(C.byref(m), 8, 0.5, 1.0, dummy, dummy, dummy, None) == cl.CL_ERR_ARG
    assert b"1 or 2 fields" in lib.cl_last_error(None)


def _unbound_lattice(N, precision=cl.CL_FP64):
    """A Lattice object with no handle: the binding's own checks run, and any
    call that got past them would fail on the NULL handle, not on memory."""
    lat = object.__new__(cl.Lattice)
    lat.h, lat.N, lat.grid = None, N, cl.make_grid(N, 0.5, 0.01, precision=precision)
    return lat


@pytest.mark.parametrize("buf", ["short", "long", "float32", "strided"])
def test_field_copies_reject_buffers_of_the_wrong_size_or_type(buf):
    """get_field / set_field copy exactly N^3 doubles; any other buffer is
    refused before the library is called, so a short host array or device
    tensor never takes a copy of N^3 elements."""
    N = 4
    a = {"short": np.zeros(N ** 3 - 1), "long": np.zeros(N ** 3 + 1), "float32": np.zeros(N ** 3, np.float32),
         "strided": np.zeros(2 * N ** 3)[::2]}[buf]
    lat = _unbound_lattice(N)
    with pytest.raises(ValueError):
        lat.get_field(cl.FIELD(0), a)
    if buf != "float32" and buf != "strided":  # set_field converts dtype and layout of host arrays
        with pytest.raises(ValueError):
            lat.set_field(cl.FIELD(0), a)


def test_field_copies_reject_short_tensors():
    torch = pytest.importorskip("torch")
    lat = _unbound_lattice(4)
    for t in (torch.zeros(63, dtype=torch.float64), torch.zeros(64, dtype=torch.float32),
              torch.zeros(128, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            lat.get_field(cl.FIELD(0), t)
        with pytest.raises(ValueError):
            lat.set_field(cl.FIELD(0), t)


@pytest.mark.parametrize("precision", [cl.CL_FP32, cl.CL_FP64])
def test_stored_copies_take_the_handle_precision(precision):
    lat = _unbound_lattice(4, precision)
    other = np.float64 if precision == cl.CL_FP32 else np.float32
    for a in (np.zeros(64, other), np.zeros(63, np.float32 if precision == cl.CL_FP32 else np.float64)):
        with pytest.raises(ValueError):
            lat.get_stored(cl.FIELD(0), a)
        with pytest.raises(ValueError):
            lat.set_stored(cl.FIELD(0), a, 0.0)


@pytest.mark.parametrize("bad", ["n", "null_q", "model", "pexp", "integrator", "size", "size_cap", "q_negative",
                                 "q_nan"])
def test_ensemble_init_rejects_bad_arguments_before_any_device_work(bad):
    """ensemble_init refuses, with CL_ERR_ARG and a reason, what the header lists:
    n < 1, NULL arrays, a model other than the two-field pexp = 2 scalar model,
    an integrator other than VV2/VV4, N outside the multiples of 32 in [32, 1024],
    q < 0 or NaN."""
    lib = cl.load()
    n = 2
    model = cl.make_model(n_fields=2, pexp=2)
    grid = cl.make_grid(32, 0.5, 0.01, "vv4", cl.CL_FP32)
    q = np.array([1.0, 2.0])
    Ns = np.array([32, 64], dtype=np.int32)
    seeds = np.array([1, 2], dtype=np.uint64)
    if bad == "n":
        n = 0
    if bad == "model":
        model.kind = cl.CL_MODEL_U1
    if bad == "pexp":
        model.pexp = 4
    if bad == "integrator":
        grid.integrator = cl.CL_INT_LF
    if bad == "size":
        Ns[1] = 48
    if bad == "size_cap":
        Ns[1] = 2048
    if bad == "q_negative":
        q[0] = -1.0
    if bad == "q_nan":
        q[1] = np.nan
    pq = None if bad == "null_q" else q.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    st = lib.ensemble_init(n, C.byref(model), pq, Ns.ctypes.data_as(C.POINTER(C.c_int32)),
                           seeds.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(grid), C.byref(cl.make_init()), None,
                           C.byref(h))
    assert st == cl.CL_ERR_ARG and not h.value
    assert b"ensemble_init" in lib.cl_last_error(None)


def test_ensemble_null_handles_are_rejected():
    lib = cl.load()
    out = C.c_void_p()
    assert lib.ensemble_member(None, 0, C.byref(out)) == cl.CL_ERR_ARG
    assert lib.ensemble_evolve(None, 1) == cl.CL_ERR_ARG
    assert lib.ensemble_observe(None, 0.0, None, None) == cl.CL_ERR_ARG
    assert lib.ensemble_destroy(None) == cl.CL_OK
