"""Pins of the oracle's initial conditions (section 7), spectra (sections 3.1,
4.4.2) and random draws (Philox4x32-10)."""
import numpy as np
import pytest

from oracle import ScalarLattice, ScalarModel, SU2Lattice, SU2Model, U1Lattice, U1Model, philox
from oracle.ic import mode_map, scalar_ic, su2_ic, u1_ic
from oracle.spectra import dft_forward, shell_bins, spectrum


def test_philox_known_answers():
    rows = [l.split() for l in open("tests/golden/philox4x32_10_kat.txt") if not l.startswith("#") and l.strip()]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        ctr, key, out = v[:4], v[4:6], v[6:10]
        got = philox.philox4x32_10([np.array([c]) for c in ctr], key)
        assert [int(g[0]) for g in got] == out


def test_mode_map_is_a_hermitian_pairing():
    N = 6
    lin, conj, selfc, zero, kabs = mode_map(N)
    # every half-layout source index is used by a mode and its conjugate, or by one self-conjugate mode
    assert selfc.sum() == 8  # components in {0, N/2}
    for z in range(N):
        for y in range(N):
            for x in range(N):
                nz, ny, nx = (-z) % N, (-y) % N, (-x) % N
                assert lin[z, y, x] == lin[nz, ny, nx]
                if not selfc[z, y, x]:
                    assert conj[z, y, x] != conj[nz, ny, nx]


def _scalar_setup(N=16, kIR=0.5, seed=3):
    dx = 2 * np.pi / (kIR * N)
    m = ScalarModel(N=N, Ns=2, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, q=2.0)
    phi, pi, _ = scalar_ic(m, kIR, [1.0, 0.0], [0.0, 0.0], seed=seed, omega_over_fstar=0.1)
    return m, phi, pi, dx


def test_vacuum_fluctuations_have_the_target_mode_variance():
    """Per shell, <|dphi(n~)|^2> / ((w*/f*)^2 (N/dx)^3 / (2 a^2 w_k)) -> 1 within
    its sampling error (|dphi|^2 is exponentially distributed, section 7.1),
    and <|dphi'(n~) + H dphi(n~)|^2> carries the extra w_k^2."""
    N, kIR = 16, 0.5
    m, phi, pi, dx = _scalar_setup(N, kIR)
    lin, conj, selfc, zero, nabs = mode_map(N)
    k = kIR * nabs
    for i, m2 in enumerate([1.0 + 0.0, 2.0 * 1.0]):  # d2V/dphi2 = lam + q chi^2, d2V/dchi2 = q phi^2
        w = np.sqrt(k ** 2 + m2)
        T = np.where(zero, 1.0, 0.1 ** 2 * (N / dx) ** 3 / (2 * w))
        P = np.abs(dft_forward(phi[i] - phi[i].mean())) ** 2 / T
        Pd = np.abs(dft_forward(pi[i])) ** 2 / (T * w * w)
        b, _, nb = shell_bins(N)
        for s in range(1, nb):
            sel = (b == s) & ~selfc
            c = sel.sum()
            if c < 60:
                continue
            tol = 5.0 * np.sqrt(2.0 / c)
            assert abs(P[sel].mean() - 1) < tol, (i, s, P[sel].mean())
            assert abs(Pd[sel].mean() - 1) < tol, (i, s, Pd[sel].mean())
    assert abs(phi[0].mean() - 1.0) < 1e-14 and abs(phi[1].mean()) < 1e-14


def test_self_conjugate_modes_have_the_target_variance():
    """The modes equal to their own conjugate (components in {0, N/2}) are real;
    drawn as sqrt(2) Re of a complex draw they keep the target variance of the
    other modes (reading 9 of the design).  Over 60 seeds the mean of
    |dphi(n~)|^2 / T over the seven nonzero such modes is 1 within its sampling
    error (chi-squared with one degree of freedom: standard error
    sqrt(2 / (7 x 60)) = 0.069), and likewise for the momenta."""
    N, kIR, seeds = 8, 0.5, 60
    dx = 2 * np.pi / (kIR * N)
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, q=0.0)
    lin, conj, selfc, zero, nabs = mode_map(N)
    sel = selfc & ~zero
    assert sel.sum() == 7
    w = np.sqrt((kIR * nabs[sel]) ** 2 + 1.0)  # V'' = lam for V = phi^2 / 2
    T = 0.1 ** 2 * (N / dx) ** 3 / (2 * w)
    rf, rp = [], []
    for seed in range(seeds):
        phi, pi, _ = scalar_ic(m, kIR, [1.0], [0.0], seed=seed, omega_over_fstar=0.1)
        rf.append(np.abs(dft_forward(phi[0] - phi[0].mean()))[sel] ** 2 / T)
        rp.append(np.abs(dft_forward(pi[0]))[sel] ** 2 / (T * w * w))
    se = np.sqrt(2.0 / (7 * seeds))
    assert abs(np.mean(rf) - 1.0) < 4 * se, np.mean(rf)
    assert abs(np.mean(rp) - 1.0) < 4 * se, np.mean(rp)



def test_vacuum_draw_in_an_expanding_background():
    """At a = 2, alpha = 1/2 and a program Hubble rate H of order one (section 7.1):
      - the homogeneous momentum is pi = a^{3-alpha} phi' (section 4.2.3), so the
        state without fluctuations has E_K = phi'^2/(2 a^{2 alpha}) (section 4.4.1);
      - H is the one of the evolution's Hubble constraint for that state, H = b/a;
      - |dphi(n~)|^2 averages (w*/f*)^2 (N/dx)^3/(2 a^2 w_k), w_k = sqrt(k^2 + a^2 m^2);
      - dphi'(n~) = -H dphi(n~) + a^{alpha-1} i w_k (l - r)/sqrt(2) with the second
        part uncorrelated with dphi, so sum Re[dphi* dphi'] / sum |dphi|^2 -> -H and
        |dphi' + H dphi|^2 averages a^{2(alpha-1)} w_k^2 times the field's variance.
    Each mean is taken over the ~2000 independent modes of a 16^3 draw and held to
    four standard errors."""
    N, kIR, a, alpha, fmp2 = 16, 0.1, 2.0, 0.5, 6.0
    dx = 2 * np.pi / (kIR * N)
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=alpha, fmp2=fmp2, lam=1.0, q=0.0)  # m^2 = lam = 1
    phibar, dphibar = 1.0, 0.3
    phi0, pi0, _ = scalar_ic(m, kIR, [phibar], [dphibar], seed=0, omega_over_fstar=0.1, a=a, fluctuations=False)
    hom = ScalarLattice(m, phi0, pi0, a=a)
    assert abs(hom.energies()[0] / (dphibar ** 2 / (2 * a ** (2 * alpha))) - 1) < 1e-13
    H = np.sqrt(hom.hubble_rhs()) / a
    assert H > 1.0
    lin, conj, selfc, zero, nabs = mode_map(N)
    sel = ~selfc & ~zero
    M = sel.sum() / 2  # independent modes: n~ and -n~ carry conjugate values
    w = np.sqrt((kIR * nabs) ** 2 + a * a * 1.0)
    T = 0.1 ** 2 * (N / dx) ** 3 / (2 * a * a * w)
    phi, pi, _ = scalar_ic(m, kIR, [phibar], [dphibar], seed=11, omega_over_fstar=0.1, a=a)
    F = dft_forward(phi[0] - phibar)
    Fd = dft_forward(pi[0] / a ** (3.0 - alpha) - dphibar)
    r_var = np.mean(np.abs(F[sel]) ** 2 / T[sel])
    assert abs(r_var - 1) < 4 / np.sqrt(M), r_var
    corr = np.sum((np.conj(F) * Fd).real[sel]) / np.sum(np.abs(F[sel]) ** 2)
    se = np.max(a ** (alpha - 1) * w) / np.sqrt(2 * M)
    assert abs(corr + H) < 4 * se, (corr, -H, se)
    r_mom = np.mean(np.abs(Fd + H * F)[sel] ** 2 / (a ** (2 * (alpha - 1)) * w * w * T)[sel])
    assert abs(r_mom - 1) < 4 / np.sqrt(M), r_mom

def test_ic_is_deterministic_in_the_seed():
    _, a, _, _ = _scalar_setup(seed=11)
    _, b, _, _ = _scalar_setup(seed=11)
    _, c, _, _ = _scalar_setup(seed=12)
    assert np.array_equal(a, b) and not np.allclose(a, c)


def test_spectrum_parseval_and_plane_wave():
    """Sum over shells of count * <|f(n~)|^2> / N^6 equals <f^2> (DFT identity of
    section 3.1); a plane wave puts all its power in one shell."""
    N, kIR = 12, 0.3
    dx = 2 * np.pi / (kIR * N)
    f = np.random.default_rng(0).standard_normal((N, N, N))
    k, D, cnt = spectrum(f, dx, kIR)
    with np.errstate(divide="ignore", invalid="ignore"):
        P = np.where(k > 0, D * 2 * np.pi ** 2 / k ** 3 / (dx / N) ** 3, 0.0)
    F0 = abs(dft_forward(f)[0, 0, 0]) ** 2
    assert abs((np.sum(P * cnt) + F0) / N ** 6 - (f ** 2).mean()) < 1e-12
    x = np.arange(N)
    wave = np.cos(2 * np.pi * 3 * x / N)[None, None, :] * np.ones((N, N, 1))
    k, D, cnt = spectrum(wave, dx, kIR)
    assert np.count_nonzero(D > 1e-20) == 1 and D[3] > 0
    assert 3 * kIR <= k[3] < 4 * kIR  # k of a shell is k_IR times the mean |n~| of its modes
    assert cnt.sum() == N ** 3


def test_ic_spectrum_follows_vacuum_power_spectrum():
    """Delta(k) of the initial fluctuations scatters around the continuum vacuum
    spectrum k^3/(2 pi^2) (w*/f*)^2 / (2 w_k) (section 7.1)."""
    N, kIR = 16, 0.5
    m, phi, pi, dx = _scalar_setup(N, kIR)
    k, D, cnt = spectrum(phi[1], dx, kIR)
    w = np.sqrt(k ** 2 + 2.0)
    target = k ** 3 / (2 * np.pi ** 2) * 0.1 ** 2 / (2 * w)
    sel = cnt > 100
    ratio = D[sel] / target[sel]
    assert np.all(np.abs(ratio - 1) < 6 * np.sqrt(2.0 / cnt[sel]) + 0.05)


def test_u1_ic_has_zero_charge_and_satisfies_gauss():
    N = 12
    m = U1Model(N=N, dx=0.5, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=1.0, kappa=1.0)
    phi, pi, th, piA, dx = u1_ic(m, 2 * np.pi / (N * 0.5), [0.0, 0.0], [0.0, 0.0], seed=21, omega_over_fstar=1.0)
    rho = phi[0] * pi[1] - phi[1] * pi[0]
    assert abs(rho.sum()) < 1e-12 * np.abs(rho).sum()
    lat = U1Lattice(m, phi, pi, th, piA)
    assert lat.gauss() < 1e-14
    assert np.all(th == 0.0)
    # both components fluctuate with the same statistics
    assert 0.5 < phi[0].var() / phi[1].var() < 2.0



def _higgs_curvature(stored, c, lam, v2, h=1e-3):
    """d^2V/dchi_c^2 of V = (lam/4)(|Phi|^2 - v2)^2 along the canonical component
    chi_c = sqrt(2) Phi_c (|Phi|^2 = sum of the stored components squared), by
    central differences of the potential itself."""
    def V(chi):
        f = np.array(stored, dtype=float)
        f[c] = chi / np.sqrt(2.0)
        return 0.25 * lam * (np.sum(f * f) - v2) ** 2
    x0 = np.sqrt(2.0) * stored[c]
    return (V(x0 + h) - 2 * V(x0) + V(x0 - h)) / (h * h)


@pytest.mark.parametrize("sector", ["u1", "su2"])
def test_charged_draws_follow_the_canonical_curvature(sector):
    """Charged scalars (sections 5, 6, 7.2) are stored as components Phi_c with
    |Phi|^2 = sum_c Phi_c^2 and canonical fields chi_c = sqrt(2) Phi_c.  Each
    canonical component fluctuates like a real scalar (section 7.1) whose mass is
    the potential's curvature along it, so the stored component's per-mode
    variance is (w*/f*)^2 (N/dx)^3 / (4 a^2 w_k) with w_k^2 = k^2 + a^2 V''(chi_c),
    V'' taken here by finite differences of the Higgs potential.  The U(1)
    homogeneous value is given canonically, so its stored mean is phibar/sqrt(2).
    Held to four standard errors over the ~2000 independent modes of 16^3 (the
    U(1) draw's equal moduli double the per-mode variance of |dphi|^2)."""
    N, kIR, lam, v2 = 16, 0.1, 1.0, 1.0
    dx = 2 * np.pi / (kIR * N)
    lin, conj, selfc, zero, nabs = mode_map(N)
    sel = ~selfc & ~zero
    M = sel.sum() / 2
    if sector == "u1":
        m = U1Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=lam, v2=v2, e=1.0, kappa=1.0, pot=0)
        pb = [1.6, 0.4]
        phi = u1_ic(m, kIR, pb, [0.0, 0.0], seed=31, omega_over_fstar=0.1)[0]
        stored_mean = [x / np.sqrt(2.0) for x in pb]
        sigma = np.sqrt(2.0)
    else:
        m = SU2Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=lam, v2=v2, g=1.0, kappa=1.0, pot=0)
        stored_mean = [1.1, 0.0, 0.3, 0.0]
        phi = su2_ic(m, kIR, stored_mean, [0.0] * 4, seed=31, omega_over_fstar=0.1)[0]
        sigma = 1.0
    assert np.allclose([p.mean() for p in phi], stored_mean, rtol=0, atol=1e-13)
    for c in range(len(stored_mean)):
        m2 = _higgs_curvature(stored_mean, c, lam, v2)
        w = np.sqrt((kIR * nabs) ** 2 + abs(m2))
        T = 0.1 ** 2 * (N / dx) ** 3 / (4 * w)
        r = np.mean(np.abs(dft_forward(phi[c] - phi[c].mean()))[sel] ** 2 / T[sel])
        assert abs(r - 1) < 4 * sigma / np.sqrt(M), (c, m2, r)


@pytest.mark.parametrize("sector", ["u1", "su2"])
def test_charged_draws_carry_the_hubble_term(sector):
    """dphi' = -H dphi + (a part uncorrelated with dphi) for every stored component
    of a charged scalar (section 7.1, with the charged fields of sections 7.2 and
    6), H the program Hubble rate of the homogeneous state: H = b/a with b^2 =
    (f*/m_p)^2 a^{2(alpha+1)} (sum of the lattice energies of that state) / 3
    (section 4.1), the energies taken by the sector's energy functional.  The
    homogeneous velocity carries most of the energy, so its kinetic term decides H."""
    N, kIR, a, alpha, fmp2 = 16, 0.1, 1.5, 0.5, 6.0
    dx = 2 * np.pi / (kIR * N)
    lin, conj, selfc, zero, nabs = mode_map(N)
    sel = ~selfc & ~zero
    M = sel.sum() / 2
    if sector == "u1":
        m = U1Model(N=N, dx=dx, alpha=alpha, fmp2=fmp2, lam=1.0, v2=1.0, e=1.0, kappa=1.0, pot=0)
        pb, db = [1.2, 0.3], [1.5, -0.8]
        draw = lambda seed, fs: u1_ic(m, kIR, pb, db, seed=seed, omega_over_fstar=0.1, a=a, fluct_scale=fs)
        hom = draw(0, 0.0)
        E = U1Lattice(m, hom[0], hom[1], hom[2], hom[3], a=a).energies()
        mean_phi, mean_dphi = [x / np.sqrt(2.0) for x in pb], [x / np.sqrt(2.0) for x in db]
    else:
        m = SU2Model(N=N, dx=dx, alpha=alpha, fmp2=fmp2, lam=1.0, v2=1.0, g=1.0, kappa=1.0, pot=0)
        pb = [0.9, 0.0, 0.2, 0.0]
        db = [1.2 * x for x in pb]  # parallel to Phi: no homogeneous charge
        draw = lambda seed, fs: su2_ic(m, kIR, pb, db, seed=seed, omega_over_fstar=0.1, a=a, fluct_scale=fs)
        hom = draw(0, 0.0)
        E = SU2Lattice(m, hom[0], hom[1], hom[2], hom[3], a=a).energies()
        mean_phi, mean_dphi = pb, db
    H = np.sqrt(fmp2 / 3.0 * a ** (2 * (alpha + 1)) * E.sum()) / a
    assert H > 1.5
    phi, pi = draw(7, 1.0)[:2]
    num = den = 0.0
    for c in range(len(pb)):
        F = dft_forward(phi[c] - mean_phi[c])
        Fd = dft_forward(pi[c] / a ** (3.0 - alpha) - mean_dphi[c])
        num += np.sum((np.conj(F) * Fd).real[sel])
        den += np.sum(np.abs(F[sel]) ** 2)
    w_max = np.sqrt((kIR * nabs.max()) ** 2 + 4.0)
    se = a ** (alpha - 1) * w_max / np.sqrt(2 * M * len(pb))
    assert abs(num / den + H) < 4 * se, (num / den, -H, se)


def test_scalar_draw_follows_the_potential_curvature():
    """Each scalar fluctuates with the curvature of V = (lam/p)|phi|^p + (q/2) phi^2 chi^2
    (section 8.1) along itself at the homogeneous values (section 7.1), here with
    both homogeneous values non-zero so that the interaction enters both
    curvatures; V'' by finite differences of the potential."""
    N, kIR, lam, q, p = 16, 0.1, 1.0, 3.0, 4
    dx = 2 * np.pi / (kIR * N)
    m = ScalarModel(N=N, Ns=2, pexp=p, dx=dx, alpha=0.0, fmp2=0.0, lam=lam, q=q)
    pb = [0.5, 1.0]
    phi = scalar_ic(m, kIR, pb, [0.0, 0.0], seed=17, omega_over_fstar=0.1)[0]
    lin, conj, selfc, zero, nabs = mode_map(N)
    sel = ~selfc & ~zero
    M = sel.sum() / 2

    def V(f0, f1):
        return lam / p * abs(f0) ** p + 0.5 * q * f0 * f0 * f1 * f1

    h = 1e-3
    curv = [(V(pb[0] + h, pb[1]) - 2 * V(*pb) + V(pb[0] - h, pb[1])) / h ** 2,
            (V(pb[0], pb[1] + h) - 2 * V(*pb) + V(pb[0], pb[1] - h)) / h ** 2]
    for i in range(2):
        w = np.sqrt((kIR * nabs) ** 2 + curv[i])
        T = 0.1 ** 2 * (N / dx) ** 3 / (2 * w)
        r = np.mean(np.abs(dft_forward(phi[i] - pb[i]))[sel] ** 2 / T[sel])
        assert abs(r - 1) < 4 / np.sqrt(M), (i, curv[i], r)


@pytest.mark.parametrize("N", [6, 12, 16])
def test_shell_count_is_the_number_of_shells(N):
    """|n~| runs up to sqrt(3) N/2 (the corner mode), so there are
    floor(sqrt(3) N/2) + 1 shells [b, b+1), every one of them occupied, and the
    spectrum reports each."""
    b, nabs, nb = shell_bins(N)
    assert nb == int(np.floor(np.sqrt(3) * N / 2 + 1e-12)) + 1
    k, D, cnt = spectrum(np.random.default_rng(N).standard_normal((N, N, N)), 1.0, 1.0)
    assert len(cnt) == nb and np.all(cnt > 0) and cnt.sum() == N ** 3

@pytest.mark.parametrize("N", [4, 8])
def test_isqrt_bins_are_exact(N):
    b, nabs, nb = shell_bins(N)
    assert np.all(b * b <= nabs ** 2 + 1e-9) and np.all((b + 1) ** 2 > nabs ** 2 - 1e-9)
