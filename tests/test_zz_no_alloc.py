"""lattice_energies_noalloc: the entry point for callers that cannot call
cudaMalloc (programs whose own memory pool owns the GPU, loops that must never
enter the allocator).  It must give the energies and means of the oracle and of
lattice_measure_means, call after call, while using only its fixed device
scratch array.

This file is named so that pytest collects it last; it passes alone in a fresh
process (the first call performs the per-device set-up) and after the rest.
"""
import ctypes
import math

import numpy as np
import pytest

import paper_2006_15122_gb300 as cl
from oracle import ScalarLattice, ScalarModel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nf,pexp", [(1, 2), (1, 6), (2, 4)])
def test_noalloc_energies_match_oracle_and_measure_means_twice(nf, pexp):
    import torch

    N, kIR, lam, q = 48, 0.5, 1.0, 3.0
    dx = 2 * math.pi / (kIR * N)
    model = cl.make_model(n_fields=nf, pexp=pexp, lam=lam, q=q, omega_over_fstar=0.05, fstar_over_mp=1.0, alpha=1.0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, 0.01, "vv4", cl.CL_FP64),
                     cl.make_init(phi0=(1.0, 0.1)[:nf], seed=13))
    om = ScalarModel(N=N, Ns=nf, pexp=pexp, dx=dx, alpha=1.0, fmp2=1.0, lam=lam, q=q)
    out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
    phi = torch.empty((nf, N, N, N), dtype=torch.float64, device="cuda")
    pi = torch.empty((nf, N, N, N), dtype=torch.float64, device="cuda")
    before = torch.cuda.memory_allocated()
    for call in range(2):
        lat.evolve(3)  # a different state for each call
        mm = lat.measure_means()
        for i in range(nf):
            lat.get_field(cl.FIELD(i), phi[i])
            lat.get_field(cl.MOMENTUM(i), pi[i])
        out.fill_(float("nan"))
        cl.energies_noalloc(model, N, kIR, mm["a"], phi, pi, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o)), (call, o)
        # the oracle's energies of the same arrays (FP64 parity tolerance)
        ref = ScalarLattice(om, phi.cpu().numpy(), pi.cpu().numpy(), a=mm["a"])
        E = ref.energies()  # E_K[0..1], E_G[0..1], E_V terms
        assert np.allclose(o[0:nf], E[0:nf], rtol=1e-12, atol=0.0), (call, o, E)
        assert np.allclose(o[2:2 + nf], E[2:2 + nf], rtol=1e-12, atol=0.0), (call, o, E)
        assert np.allclose(o[4:6], E[4:6], rtol=1e-12, atol=1e-300), (call, o, E)
        means = ref.phi.reshape(nf, -1).mean(axis=1)
        dev = ref.phi.reshape(nf, -1) - means[:, None]
        var = (dev ** 2).mean(axis=1)
        assert np.allclose(o[6:6 + nf], means, rtol=1e-12, atol=0.0), (call, o, means)
        assert np.allclose(o[8:8 + nf], var, rtol=1e-10, atol=0.0), (call, o, var)
        # and lattice_measure_means of the handle that produced them
        mref = np.array(mm["EK"][:nf] + mm["EG"][:nf] + mm["mean"][:nf] + mm["var"][:nf])
        mgot = np.concatenate([o[0:nf], o[2:2 + nf], o[6:6 + nf], o[8:8 + nf]])
        assert np.allclose(mgot, mref, rtol=1e-10, atol=0.0), (call, mgot, mref)
        if nf == 1:  # the slots of an absent second field are exactly zero
            assert o[1] == 0.0 and o[3] == 0.0 and o[5] == 0.0 and o[7] == 0.0 and o[9] == 0.0, o
    assert torch.cuda.memory_allocated() == before
    lat.close()


def test_noalloc_variance_of_a_large_mean_keeps_its_digits():
    """phi = 1 + 1e-6 fluctuations: the variance (1e-12) must not be lost to the
    cancellation of <phi^2> - <phi>^2 (about 1e-16 relative of <phi^2>)."""
    import torch

    N, kIR = 32, 0.5
    model = cl.make_model(n_fields=1, pexp=2, lam=1.0, omega_over_fstar=1.0, fstar_over_mp=0.0)
    rng = np.random.default_rng(5)
    f = 1.0 + 1e-6 * rng.standard_normal((N, N, N))
    p = 1e-3 * rng.standard_normal((N, N, N))
    phi = torch.as_tensor(f, device="cuda").contiguous()
    pi = torch.as_tensor(p, device="cuda").contiguous()
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    for _ in range(2):
        cl.energies_noalloc(model, N, kIR, 1.0, phi, pi, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert abs(o[6] - f.mean()) < 1e-15
        assert abs(o[8] - f.var()) < 1e-10 * f.var(), (o[8], f.var())


def test_noalloc_rejects_sizes_beyond_its_limit_and_short_buffers():
    import torch

    model = cl.make_model(n_fields=1)
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    lib = cl.load()
    ptr = ctypes.c_void_p(t.data_ptr())
    # straight through the C ABI: the library itself refuses N beyond its limit
    st = lib.lattice_energies_noalloc(ctypes.byref(model), 4096, 0.5, 1.0, ptr, ptr, ptr, None)
    assert st == cl.CL_ERR_ARG and b"2048" in lib.cl_last_error(None)
    with pytest.raises(ValueError):
        cl.energies_noalloc(model, 4, 0.5, 1.0, t, t, t)  # phi needs 64 elements
