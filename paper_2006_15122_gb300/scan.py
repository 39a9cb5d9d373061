"""Parameter scans over the resonance coupling q of the two-field model
V = phi^2/2 + (q*/2) phi^2 chi^2, q* = 4q (section 8.1): a batched ensemble of lattices
observed at uniform time slices, a surrogate network fitted to those
observations, and the one-lattice-at-a-time method the surrogate stands in for.

Every step runs in the library (ensemble_*, lattice_*, surrogate_* through the
C ABI); this module only sequences the calls, arranges the observations as
training pairs (log10 q, t) -> CL_OBS_SIZE observables, and scores
predictions against fresh lattice runs.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import (CL_FP32, CL_INT_VV4, CL_OBS_SIZE, Ensemble, Lattice, Surrogate, make_grid, make_init,
               make_model)


@dataclass
class ScanSpec:
    """Model, grid and observation schedule shared by every run of a scan."""
    fstar_over_mp: float = 1.396
    omega_over_fstar: float = 5.13e-6
    kIR: float = 0.1
    # Slices one inflaton half-period apart (pi in program units, where the inflaton
    # mass is 1): phi^2, and with it w, the energy split and the burst-wise chi
    # production, is sampled at one phase of the oscillation, so each observable
    # varies slowly from slice to slice.  Slices a quarter period apart would
    # alternate between kinetic and potential domination (w near +1, then -1).
    # dt = pi/1571 is the VV4-stable step for q* <= 4e5 (omega_chi dt = 1.264 < 1.573).
    dt: float = math.pi / 1571
    integrator: int = CL_INT_VV4
    precision: int = CL_FP32
    sizes: tuple = (32, 64, 96)
    steps_per_slice: int = 1571  # 64 slices to t = 64 pi = 201, past the q = 1e4 workload's horizon t = 100
    n_slices: int = 64
    phi0: float = 1.0
    nmin: int = field(default=0)

    def __post_init__(self):
        if not self.nmin:
            self.nmin = min(self.sizes)

    @property
    def kmax(self):
        """Upper end of the observed spectrum: the axis Nyquist momentum of the smallest lattice."""
        return 0.5 * self.nmin * self.kIR

    def times(self):
        return self.dt * self.steps_per_slice * np.arange(1, self.n_slices + 1)

    def model(self, q=0.0):
        """Program-unit model of resonance parameter q = g^2 Phi^2 / (4 m^2): with
        omega_star = m and phi_star = Phi the coupling of (1/2) q* phi^2 chi^2 is
        q* = g^2 Phi^2 / m^2 = 4 q (section 8.1)."""
        return make_model(n_fields=2, pexp=2, lam=1.0, q=4.0 * q, omega_over_fstar=self.omega_over_fstar,
                          fstar_over_mp=self.fstar_over_mp)

    def grid(self, N):
        return make_grid(N, self.kIR, self.dt, self.integrator, self.precision)

    def init(self, seed=0):
        return make_init(phi0=(self.phi0, 0.0), seed=seed)


def log_uniform_q(n, lo, hi, seed):
    """n couplings log-uniform in [lo, hi] (numpy PCG64 stream of `seed`)."""
    return 10.0 ** np.random.default_rng(seed).uniform(math.log10(lo), math.log10(hi), n)


def cycle_sizes(n, sizes):
    return [sizes[i % len(sizes)] for i in range(n)]


def ensemble_observations(spec, qs, Ns, seeds, autotune=True, stream=None):
    """Observations of a batched ensemble at spec.n_slices uniform slices
    (qs: resonance parameters q, see ScanSpec.model).

    Returns (obs of shape (n, n_slices, CL_OBS_SIZE), times, info) where info
    holds the wall-clock seconds of initialisation, tuning and evolution (each
    phase ends synchronized) and the tile shape used.  An empty run list (a rank
    whose partition() block is empty) gives no observations and launches nothing."""
    if len(qs) == 0:
        return (np.zeros((0, spec.n_slices, CL_OBS_SIZE), dtype=np.float32), spec.times(),
                {"init_s": 0.0, "tune_s": 0.0, "evolve_observe_s": 0.0, "tile": None, "candidates": []})
    t0 = time.perf_counter()
    ens = Ensemble(spec.model(), 4.0 * np.asarray(qs, dtype=np.float64), Ns, seeds, spec.grid(spec.nmin),
                   spec.init(), stream=stream)
    t1 = time.perf_counter()
    try:
        tuned = ens.autotune() if autotune else []
        t2 = time.perf_counter()
        obs = np.zeros((len(qs), spec.n_slices, CL_OBS_SIZE), dtype=np.float32)
        times = np.zeros(spec.n_slices)
        for j in range(spec.n_slices):
            ens.evolve(spec.steps_per_slice)
            obs[:, j, :], times[j] = ens.observe(spec.kmax)
        t3 = time.perf_counter()
        info = {"init_s": t1 - t0, "tune_s": t2 - t1, "evolve_observe_s": t3 - t2, "tile": ens.tile(),
                "candidates": tuned}
    finally:
        ens.close()
    return obs, times, info


def plain_observations(spec, q, N, seed, stream=None):
    """The same observations from one lattice evolved on its own (the method
    without batching): (obs (n_slices, CL_OBS_SIZE), times)."""
    m = spec.model(q)
    lat = Lattice(m, spec.grid(N), spec.init(seed), stream=stream)
    try:
        obs = np.zeros((spec.n_slices, CL_OBS_SIZE), dtype=np.float32)
        times = np.zeros(spec.n_slices)
        for j in range(spec.n_slices):
            lat.evolve(spec.steps_per_slice)
            obs[j], times[j] = lat.observe(spec.kmax)
    finally:
        lat.close()
    return obs, times


def partition(n, world, rank):
    """The runs of an n-run scan that rank `rank` of `world` evolves: a
    contiguous block, the first n % world ranks one run longer.  The blocks
    cover 0..n-1 once, in order."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return list(range(lo, lo + base + (1 if rank < extra else 0)))


def gather_runs(local, n, dist=None, device="cpu"):
    """All ranks' observations of their partition() blocks, assembled in run
    order on every rank: local has shape (len(block), ...).  One all_gather of
    equally padded blocks (NCCL on GPUs, gloo on CPU ranks); without a process
    group the local array is the whole scan."""
    local = np.ascontiguousarray(local)
    if dist is None:
        if local.shape[0] != n:
            raise ValueError("without a process group the local block is the whole scan: %d rows, not %d"
                             % (local.shape[0], n))
        return local
    import torch

    world = dist.get_world_size()
    rows = -(-n // world)
    pad = np.full((rows,) + local.shape[1:], np.nan, dtype=local.dtype)
    pad[:local.shape[0]] = local
    t = torch.from_numpy(pad).to(device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    out = [parts[r].cpu().numpy()[:len(partition(n, world, r))] for r in range(world)]
    return np.concatenate(out, axis=0)


def training_pairs(qs, times, obs):
    """(log10 q, t) -> observables, one row per run and slice."""
    n, S = len(qs), len(times)
    X = np.stack([np.repeat(np.log10(qs), S), np.tile(times, n)], axis=1).astype(np.float32)
    Y = obs.reshape(n * S, -1).astype(np.float32)
    ok = np.all(np.isfinite(Y), axis=1)
    return X[ok], Y[ok]


def fit_surrogate(X, Y, width=256, depth=3, epochs=200, batch=512, lr=2e-3, lr_end=2e-5, seed=0, stream=None):
    """Surrogate network fitted to (X, Y): Adam with a cosine-annealed step size,
    samples shuffled every epoch.  Returns (net, per-epoch loss, seconds)."""
    net = Surrogate(X.shape[1], Y.shape[1], width, depth, seed=seed, stream=stream)
    t0 = time.perf_counter()
    hist = net.train(X, Y, epochs=epochs, batch=batch, lr=lr, lr_end=lr_end, shuffle=True)
    return net, hist, time.perf_counter() - t0


def disagreement(pa, pb):
    """Error estimate of a surrogate answer from two independently trained
    networks: per (query, slice), the larger of |eps_a - eps_b| and |w_a - w_b|,
    the two observables gated in absolute terms (the spectrum's error is judged
    against its seed scatter, which one lattice run does not beat either)."""
    return np.maximum(np.abs(pa[..., 0] - pb[..., 0]), np.abs(pa[..., 1] - pb[..., 1]))


def answer_queries(nets, qs, times, q_range, spec, tol=0.02, frac=0.9, seeds=None, size=None, stream=None):
    """Observations at couplings qs and the given slice times, from the surrogate
    where it can be trusted and from the lattice otherwise.  A query falls back
    to a lattice run (size `size`, default the middle one of spec.sizes) when its
    q lies outside the trained range q_range, or when the two networks disagree
    by more than tol on more than 1 - frac of its slices.  The fallback runs
    evolve together as one batched ensemble with the default tile (no tuning), so
    each answer is the one a single-member ensemble of that query gives, whatever
    else fell back.  Returns (answers (Q, S, CL_OBS_SIZE), fallback mask,
    estimate (Q, S), seconds of the network queries, seconds of the fallback
    runs)."""
    Q, S = len(qs), len(times)
    X = np.stack([np.repeat(np.log10(qs), S), np.tile(times, Q)], axis=1).astype(np.float32)
    t0 = time.perf_counter()
    preds = [net.predict(X).reshape(Q, S, -1) for net in nets]
    t_query = time.perf_counter() - t0
    est = disagreement(preds[0], preds[1]) if len(preds) > 1 else np.zeros((Q, S))
    out = np.mean(preds, axis=0).astype(np.float32)
    lo, hi = q_range
    fallback = (np.asarray(qs) < lo) | (np.asarray(qs) > hi) | (np.mean(est <= tol, axis=1) < frac)
    size = size or sorted(spec.sizes)[len(spec.sizes) // 2]
    seeds = seeds if seeds is not None else list(range(2 * 10 ** 6, 2 * 10 ** 6 + Q))
    t0 = time.perf_counter()
    idx = np.nonzero(fallback)[0]
    if len(idx):
        obs, _, _ = ensemble_observations(spec, np.asarray(qs)[idx], [size] * len(idx), [seeds[i] for i in idx],
                                          autotune=False, stream=stream)
        out[idx] = obs
    t_fallback = time.perf_counter() - t0
    return out, fallback, est, t_query, t_fallback


def score(pred, ref_runs):
    """Errors of predictions against fresh lattice runs.

    pred: (Q, S, CL_OBS_SIZE); ref_runs: (Q, R, S, CL_OBS_SIZE), R seeds per
    held-out q.  The reference is the mean over seeds (of log10 Delta for the
    spectrum).  Returns absolute errors of the chi energy fraction and of w,
    relative errors |10^(pred - ref) - 1| of the spectrum, and the same measures
    for single runs around their seed mean (the seed-scatter floor)."""
    ref = np.nanmean(ref_runs, axis=1)
    e_eps = np.abs(pred[..., 0] - ref[..., 0])
    e_w = np.abs(pred[..., 1] - ref[..., 1])
    e_spec = np.abs(10.0 ** (pred[..., 2:].astype(np.float64) - ref[..., 2:]) - 1.0)
    dev = ref_runs - ref[:, None]
    f_eps = np.abs(dev[..., 0])
    f_w = np.abs(dev[..., 1])
    f_spec = np.abs(10.0 ** dev[..., 2:].astype(np.float64) - 1.0)

    def summ(a):
        a = a[np.isfinite(a)]
        return {"median": float(np.median(a)), "p95": float(np.percentile(a, 95)), "max": float(np.max(a)),
                "within_2pct": float(np.mean(a <= 0.02))}

    R = ref_runs.shape[1]
    sq = np.sqrt(R)
    return {"eps_chi_abs": summ(e_eps), "w_abs": summ(e_w), "spectrum_rel": summ(e_spec),
            "floor": {"eps_chi_abs": summ(f_eps), "w_abs": summ(f_w), "spectrum_rel": summ(f_spec)},
            # the reference's own standard error (seed scatter of one run over sqrt(R))
            "reference_stderr": {"eps_chi_abs": summ(np.nanstd(ref_runs[..., 0], axis=1) / sq),
                                 "w_abs": summ(np.nanstd(ref_runs[..., 1], axis=1) / sq),
                                 "spectrum_rel": summ(10.0 ** (np.nanstd(ref_runs[..., 2:].astype(np.float64),
                                                                         axis=1) / sq) - 1.0)}}
