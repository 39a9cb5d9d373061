"""lattice_energies_noalloc: the entry point for callers that cannot allocate
device memory (stream capture, caller-owned memory pools) must give the same
energies and means as lattice_measure_means, call after call, while using only
its fixed device scratch array.

This file is named so that pytest collects it last; it passes alone in a fresh
process (the first call performs the per-device set-up) and after the rest.
"""
import math

import numpy as np
import pytest

import paper_2006_15122_gb300 as cl

pytestmark = pytest.mark.gpu


def test_noalloc_energies_match_measure_means_twice():
    import torch

    N, kIR = 48, 0.5
    model = cl.make_model(n_fields=2, pexp=4, lam=1.0, q=3.0, omega_over_fstar=0.05, fstar_over_mp=1.0, alpha=1.0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, 0.01, "vv4", cl.CL_FP64), cl.make_init(phi0=(1.0, 0.1), seed=13))
    out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        lat.evolve(3)  # a different state for each call
        mm = lat.measure_means()
        phi = torch.empty((2, N, N, N), dtype=torch.float64, device="cuda")
        pi = torch.empty((2, N, N, N), dtype=torch.float64, device="cuda")
        for i in range(2):
            lat.get_field(cl.FIELD(i), phi[i])
            lat.get_field(cl.MOMENTUM(i), pi[i])
        out.fill_(float("nan"))
        cl.energies_noalloc(model, N, kIR, mm["a"], phi, pi, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        ref = np.array(mm["EK"][:2] + mm["EG"][:2] + mm["EV"][:2] + mm["mean"][:2] + mm["var"][:2])
        assert np.all(np.isfinite(o)), (call, o)
        # energies and means to the FP64 parity tolerance of the other tests; the
        # variance here is <phi^2> - <phi>^2 of full fields, so its rounding scales with <phi^2>
        assert np.allclose(o[:8], ref[:8], rtol=1e-12, atol=0.0), (call, o, ref)
        assert np.all(np.abs(o[8:] - ref[8:]) <= 1e-12 * np.array(mm["mean2"][:2])), (call, o, ref)
    lat.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    model = cl.make_model(n_fields=1)
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(cl.LatticeError) as e:
        cl.energies_noalloc(model, 4096, 0.5, 1.0, t, t, t)
    assert e.value.status == cl.CL_ERR_ARG and "2048" in str(e.value)
