"""Benchmark of the lattice hot path: site-updates/s of the 1024^3 two-field
preheating lattice (V = phi^2/2 + q* phi^2 chi^2/2, q = 1e5 i.e. q* = 4e5),
Yoshida VV4 steps with FP32 fluctuation arrays and FP64 means / background.

One "step" is one full VV4 time step of every site of the lattice: three
fused drift-stencil-kick-reduce passes plus the FP64 Friedmann update.  A
site-update is one site advanced one full step (all fields).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--N 1024] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank evolves its own
lattice (weak scaling, no data-path collective); value = total site-updates/s
over all ranks from the max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Workload: the throughput configuration of the paper's two-field preheating model
# (program units of sections 4.1 and 8.1; p = 2 so alpha = 0; f*/m_p and w*/f* of
# the p = 2 benchmark of section 8.2), with the time step clamped to the VV4
# stability bound of the highest chi mode (w_chi = sqrt(q*) phi = 632).
KIR = 0.1
QSTAR = 4.0e5
FSTAR_MP = 1.396
OMEGA_FSTAR = 5.13e-6
DT = 0.002
BYTES_PER_SITE_PASS = 32  # FP32: read and write delta-phi, delta-pi of two fields


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--N", type=int, default=1024)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="leave out the FP64 run that measures the FP32 error")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--with-scan", action="store_true",
                   help="append the ensemble scan (several minutes) to the single-lattice line")
    p.add_argument("--no-gauge", action="store_true", help="leave the U(1) / SU(2) pass timings out")
    p.add_argument("--gauge-only", default="", choices=["", "u1", "su2", "su2u1"],
                   help="print only the event-timed passes of one gauge sector")
    p.add_argument("--gauge-N", type=int, default=0)
    p.add_argument("--gauge-steps", type=int, default=20)
    p.add_argument("--scan", action="store_true",
                   help="time the batched ensemble + surrogate parameter scan instead of the single lattice")
    p.add_argument("--scan-runs", type=int, default=512)
    p.add_argument("--scan-slices", type=int, default=64)
    p.add_argument("--scan-steps-per-slice", type=int, default=1571)
    p.add_argument("--scan-heldout", type=int, default=64)
    p.add_argument("--scan-seeds", type=int, default=4)
    p.add_argument("--scan-plain", type=int, default=6)
    p.add_argument("--scan-epochs", type=int, default=800)
    p.add_argument("--scan-save", default="", help="write the scan's observations and answers to this .npz")
    p.add_argument("--surrogate", action="store_true",
                   help="time the surrogate's training and queries alone (scan-shaped synthetic data)")
    p.add_argument("--surrogate-epochs", type=int, default=400)
    p.add_argument("--accuracy", action="store_true",
                   help="print the Friedmann-constraint error of every integrator on the U(1) inflaton instead")
    p.add_argument("--acc-N", type=int, default=64)
    p.add_argument("--acc-eta", type=float, default=100.0)
    p.add_argument("--acc-integrators", default="lf,vv2,vv4,vv6,vv8,vv10")
    p.add_argument("--acc-model", default="u1", choices=["u1", "su2u1"],
                   help="u1: the U(1) inflaton; su2u1: the SU(2) x U(1) doublet with a singlet")
    return p.parse_args()


def workload_config(N):
    return {"workload": "%d^3 two-field phi^2 chi^2 preheating lattice, q=1e5 (q*=4e5), Yoshida VV4, "
                        "FP32 fluctuations + FP64 means/background, self-consistent expansion" % N,
            "N": N, "fields": 2, "integrator": "VV4", "kIR": KIR, "dt": DT, "qstar": QSTAR,
            "fstar_over_mp": FSTAR_MP, "omega_over_fstar": OMEGA_FSTAR,
            "state_bytes": 2 * 2 * 4 * N ** 3,
            "l2": "inputs (%.1f GB) exceed L2; no flush" % (2 * 2 * 4 * N ** 3 / 1e9)}


TRAFFIC = os.path.join(ROOT, "profiles", "scalar_pass_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2006_15122_gb300", "csrc", f) for f in ("scalar_pass.cu", "scalar_common.cuh")]


def kernel_digest():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def measured_traffic(N):
    """DRAM bytes of one pass from the committed ncu capture, scaled to N^3
    sites; None when the kernel's sources changed since the capture."""
    try:
        d = json.load(open(TRAFFIC))
    except Exception:
        return None
    if d.get("source_sha256") != kernel_digest():
        return None
    return d["dram_bytes_per_site_pass"] * N ** 3


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        """Ends the sampling, removes the sample file and summarizes it (once)."""
        if self.f.closed:
            return self.result
        text = None
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()
            self.f.flush()
            self.f.seek(0)
            text = self.f.read()
        self.f.close()
        try:
            os.unlink(self.f.name)
        except OSError:
            pass
        self.result = (self.summarize(text) if text is not None else
                       {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]})
        return self.result

    @staticmethod
    def summarize(text):
        """Median SM clock, the largest max clock and the throttle reasons seen
        Active in rows of the query above (unparsable rows are skipped)."""
        rows = [r.split(",") for r in text.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                s_, m_ = float(r[1]), float(r[2])
            except (IndexError, ValueError):
                continue
            sm.append(s_)
            smax.append(m_)
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class OracleSample:
    """The FP64 oracle as it stands on a smaller lattice of the same model
    (bounded sample of the workload), stepped on this host's cores."""

    def __init__(self, sample_N=128):
        import oracle
        from oracle.ic import scalar_ic

        self.oracle, self.N = oracle, sample_N
        dx = 2 * math.pi / (KIR * sample_N)
        om = oracle.ScalarModel(N=sample_N, Ns=2, pexp=2, dx=dx, alpha=0.0, fmp2=FSTAR_MP ** 2, lam=1.0, q=QSTAR)
        phi, pi, _ = scalar_ic(om, KIR, [1.0, 0.0], [0.0, 0.0], seed=0, omega_over_fstar=OMEGA_FSTAR)
        self.lat = oracle.ScalarLattice(om, phi, pi)
        self.lat.b = math.sqrt(self.lat.hubble_rhs())

    def step(self, n=1):
        """Seconds for n VV4 steps."""
        t0 = time.perf_counter()
        self.lat.vv_steps(self.oracle.VV4, DT, n)
        return time.perf_counter() - t0


def cpu_baseline(sample_N=128, budget_s=12.0, single_budget_s=4.0):
    """The oracle timed on a bounded sample: VV4 steps of a sample_N^3 lattice
    of the same model until about budget_s seconds of CPU work on all cores,
    then single_budget_s seconds on one thread."""
    o = OracleSample(sample_N)

    def timed(budget):
        steps, spent = 0, 0.0
        while spent < budget:
            spent += o.step(1)
            steps += 1
        return steps, spent

    steps, spent = timed(budget_s)
    lib = o.oracle.core.lib()
    cores = lib.orc_max_threads()
    lib.orc_set_threads(1)
    try:
        steps1, spent1 = timed(single_budget_s)
    finally:
        lib.orc_set_threads(cores)
    return {"value": sample_N ** 3 * steps / spent, "unit": "site-updates/s", "cores": cores,
            "kind": "oracle", "sample": "%d^3 lattice of the same model, %d VV4 steps, FP64, %.1f s"
                                        % (sample_N, steps, spent),
            "single_thread": {"value": sample_N ** 3 * steps1 / spent1, "unit": "site-updates/s", "cores": 1,
                              "sample": "%d VV4 steps, %.1f s" % (steps1, spent1)}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    N = min(args.N, 128)
    o = OracleSample(N)
    vals = []
    for i in range(args.warmup + args.steps):
        dt = o.step(1)
        if i >= args.warmup:
            vals.append(N ** 3 / dt)
    v = statistics.mean(vals)
    cfg = workload_config(args.N)
    line = {"impl": "reference", "metric": "site-updates/s", "value": v, "unit": "site-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * N ** 3 / v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"kind": "oracle", "cores": o.oracle.core.lib().orc_max_threads(), "value": v,
                             "sample": "each step: one VV4 step of a %d^3 lattice of the same model" % N},
            "e2e": {"value": v, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def scan_measurement(args, stream, dist=None):
    """Parameter scan of the two-field model over q log-uniform in [1e2, 1e5] to
    the q = 1e4 workload's horizon (t = 100):
    (i) the plain method, one lattice at a time, timed on a sample cycling
    through the sizes;
    (ii) the batched ensemble of all n runs (autotuned tiles, CUDA graphs),
    whose observations train two surrogate networks; the held-out couplings are
    then answered by the surrogate where the two networks agree within 2%, and
    by a lattice run otherwise (the fallbacks evolve together as one ensemble);
    scored against fresh lattice runs (R seeds per held-out q).
    Under torchrun the runs of both ensembles are split across the ranks (one
    block each, no exchange while they evolve) and gathered once; rank 0 trains,
    answers and scores.  Returns the line (rank 0) or None."""
    import numpy as np
    import torch

    from paper_2006_15122_gb300 import scan

    rank = dist.get_rank() if dist else 0
    world = dist.get_world_size() if dist else 1
    spec = scan.ScanSpec(steps_per_slice=args.scan_steps_per_slice, n_slices=args.scan_slices)
    n = args.scan_runs
    qs = scan.log_uniform_q(n, 1e2, 1e5, seed=1234)
    Ns = scan.cycle_sizes(n, spec.sizes)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    t_plain = None
    if rank == 0 and args.scan_plain > 0:
        # (i) plain: one lattice at a time (warm one run of each size first: plans, graphs)
        for N in spec.sizes:
            scan.plain_observations(scan.ScanSpec(sizes=spec.sizes, steps_per_slice=1, n_slices=1), qs[0], N, 0,
                                    stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.scan_plain):
            scan.plain_observations(spec, qs[i], Ns[i], i, stream)
        t_plain = (time.perf_counter() - t0) / args.scan_plain
    # (ii) batched ensemble of every run (this rank's block), gathered on every rank
    if dist:
        dist.barrier()
    blk = scan.partition(n, world, rank)
    t0 = time.perf_counter()
    obs_l, times, info = scan.ensemble_observations(spec, qs[blk], [Ns[i] for i in blk], blk, stream=stream)
    obs = scan.gather_runs(obs_l, n, dist, "cuda")
    t_ens = time.perf_counter() - t0
    # held-out couplings: fresh lattice runs (R seeds each, batched) as the reference
    Q, R = args.scan_heldout, args.scan_seeds
    qh = scan.log_uniform_q(Q, 1e2, 1e5, seed=4321)
    qr = np.repeat(qh, R)
    Nh = scan.cycle_sizes(Q * R, spec.sizes)
    blk = scan.partition(Q * R, world, rank)
    seeds = [10 ** 6 + i for i in blk]
    ref_l, _, _ = scan.ensemble_observations(spec, qr[blk], [Nh[i] for i in blk], seeds, stream=stream)
    ref = scan.gather_runs(ref_l, Q * R, dist, "cuda").reshape(Q, R, spec.n_slices, -1)
    if rank != 0:
        clocks.stop()
        return None
    X, Y = scan.training_pairs(qs, times, obs)
    nets, t_train, hists = [], 0.0, []
    for k in range(2):
        net, hist, t = scan.fit_surrogate(X, Y, epochs=args.scan_epochs, seed=k, stream=stream)
        nets.append(net)
        hists.append(hist)
        t_train += t
    # warm the query path once, then answer every held-out coupling
    nets[0].predict(X[:8])
    nets[1].predict(X[:8])
    torch.cuda.synchronize()
    ans, fb, est, t_query, t_fallback = scan.answer_queries(nets, qh, times, (qs.min(), qs.max()), spec, tol=0.02,
                                                            stream=stream)
    Xq = np.stack([np.repeat(np.log10(qh), spec.n_slices), np.tile(times, Q)], axis=1).astype(np.float32)
    pure = np.mean([net.predict(Xq).reshape(Q, spec.n_slices, -1) for net in nets], axis=0)
    clk = clocks.stop()
    err = scan.score(ans, ref)
    err_pure = scan.score(pure, ref)
    for net in nets:
        net.close()
    if args.scan_save:
        np.savez_compressed(args.scan_save, qs=qs, Ns=np.array(Ns), times=times, obs=obs, qh=qh, ref=ref, ans=ans,
                            pure=pure, fallback=fb, estimate=est)
    site_steps = sum(N ** 3 for N in Ns) * spec.steps_per_slice * spec.n_slices
    t_total = t_ens + t_train + t_query + t_fallback
    line = {
        "metric": "ensemble scan runs/hr", "value": 3600.0 * (n + Q) / t_total, "unit": "runs/hr", "n_gpus": world,
        "scaling": "strong", "higher_is_better": True, "dtype": "f32 lattice, bf16/f32 surrogate",
        "data": "synthetic",
        "config": {"workload": "%d runs of the two-field q* = 4q model, q log-uniform in [1e2, 1e5] (seed 1234), "
                               "N cycling %s, seeds 0..%d, VV4 dt %g, %d slices every %d steps (t_end %.4g), "
                               "observables eps_chi, w and the 32-point log10 chi spectrum; %d held-out q answered"
                               % (n, list(spec.sizes), n - 1, spec.dt, spec.n_slices, spec.steps_per_slice,
                                  times[-1], Q),
                   "surrogate": "two MLPs 2-256-256-256-34 GELU, BF16 tensor-core GEMMs, FP32 accumulate, Adam, "
                                "%d epochs, batch 512, %d training rows; answers where they agree within 2%% on "
                                ">= 90%% of a query's slices (eps_chi and w), a %d^3 lattice run otherwise (the "
                                "fallback runs batched in one ensemble)"
                                % (args.scan_epochs, len(X), sorted(spec.sizes)[len(spec.sizes) // 2]),
                   "heldout": "%d q log-uniform in [1e2, 1e5] (seed 4321), %d fresh seeds each" % (Q, R),
                   "parallelism": "runs split across %d ranks" % world if world > 1 else "single"},
        "value_definition": "(n training runs + Q answered queries) per hour of ensemble + training + queries + "
                            "fallback runs",
        "plain_runs_per_hr": 3600.0 / t_plain if t_plain else None,
        "batched_runs_per_hr": 3600.0 * n / t_ens,
        "batched_plus_surrogate_runs_per_hr": 3600.0 * (n + Q) / t_total,
        "speedup_vs_plain": (3600.0 * (n + Q) / t_total) / (3600.0 / t_plain) if t_plain else None,
        "fallback_queries": int(fb.sum()),
        "seconds": {"plain_per_run": t_plain, "ensemble_total": t_ens, "ensemble_init": info["init_s"],
                    "autotune": info["tune_s"], "ensemble_evolve_observe": info["evolve_observe_s"],
                    "train_two_networks": t_train, "query_all_heldout": t_query, "fallback_runs": t_fallback},
        "site_updates_per_s_batched": site_steps / info["evolve_observe_s"] if world == 1 else None,
        "tile": info["tile"],
        "train_loss_first_last": [[float(h[0]), float(h[-1])] for h in hists],
        "error": err, "error_surrogate_only": err_pure, "clocks": clk,
    }
    return line


def gauge_measurement(kind, N, steps, stream):
    """Event-timed passes of the gauge sectors on a lattice of the same shape as
    their workloads (FP32): the compact U(1) staggered leapfrog (lam = e = v = 1,
    dx = 0.5, dt = 0.1 dx; one pass per step) and the SU(2)-Higgs VV2 (one
    drift + kick per step), also with the U(1) sector and the singlet.
    Algorithmic bytes per site and pass: one read and one write of every stored
    array, 10 arrays (U(1)), 29 (SU(2)) or 37 (SU(2) x U(1) + chi) of 4 B."""
    import torch

    import paper_2006_15122_gb300 as cl

    dx = 0.5
    kIR = 2 * math.pi / (N * dx)
    if kind == "u1":
        model = cl.make_model(kind=cl.CL_MODEL_U1, lam=1.0, vev2=1.0, gauge_e=1.0, omega_over_fstar=1.0)
        init = cl.make_init(seed=7)
        integ, narr, kernel = "lf", 10, "u1_pass_kernel<float,false>"
    elif kind == "su2":
        model = cl.make_model(kind=cl.CL_MODEL_SU2, lam=1.0, vev2=1.0, gauge_e=1.0, omega_over_fstar=1.0)
        init = cl.make_init(phi0=(1.0, 0.0, 0.0, 0.0), spectrum=0)
        integ, narr, kernel = "vv2", 29, "su2_drift_kernel<float,false> + su2_kick_kernel<float,false>"
    else:  # SU(2) x U(1) + chi with the same couplings
        model = cl.make_model(kind=cl.CL_MODEL_SU2, n_fields=2, lam=1.0, vev2=1.0, gauge_e=1.0, gauge_e_u1=1.0, q=1.0,
                              omega_over_fstar=1.0)
        init = cl.make_init(phi0=(1.0, 0.0, 0.0, 0.0), spectrum=0)
        integ, narr, kernel = "vv2", 37, "su2_drift_kernel<float,true> + su2_kick_kernel<float,true>"
    lat = cl.Lattice(model, cl.make_grid(N, kIR, 0.1 * dx, integ, cl.CL_FP32), init, stream=stream)
    lat.evolve(steps)  # warm-up of the same length: the CUDA graph of `steps` steps is captured here
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.evolve(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mm = lat.measure_means()
    lat.close()
    npass = steps + (0 if kind == "u1" else 1)
    alg = 2 * narr * 4 * N ** 3
    achieved = alg / (ms / 1e3 / npass) / 1e9
    peak, _ = measured_peaks()
    return {"N": N, "integrator": integ, "steps": steps, "ms_per_step": ms / steps, "kernel": kernel,
            "bytes_per_pass": alg, "achieved_GBs": achieved, "frac": achieved / peak,
            "site_updates_per_s": N ** 3 * steps / (ms / 1e3), "gauss_violation": mm["gauss_violation"]}


def u1_inflaton_setup(p=4, M_over_mp=10.0, Lambda4_GeV4=4.3e65, qA=1.0e2):
    """Program units of the U(1)-charged monomial inflaton (section 8): the
    amplitude where slow roll ends, phi* = (M/2) asinh(sqrt(2) p m_p/M), sets
    f* = phi*; omega* = Lambda^2 M^(-p/2) phi*^((p-2)/2) gives omega*/f* =
    Lambda^2 M^(-p/2) phi*^((p-4)/2); alpha = 3(p-2)/(p+2); the program
    potential is (1/p)(2|phi|^2)^(p/2) (lam = 1) and q_A* = e^2 f*^2/omega*^2 fixes
    e.  The homogeneous start is |phi| = phi* split evenly over the two real
    components, moving radially inwards at the slow-roll velocity
    phi' = -V'/(3 H) with H^2 = (f*/m_p)^2 (phi'^2/2 + V)/3 (a = 1)."""
    m_p = 2.435e18  # reduced Planck mass in GeV
    M = M_over_mp * m_p
    phis = 0.5 * M * math.asinh(math.sqrt(2.0) * p * m_p / M)
    fmp = phis / m_p
    om = math.sqrt(Lambda4_GeV4) * M ** (-p / 2) * phis ** ((p - 4) / 2)
    e = math.sqrt(qA) * om
    alpha = 3.0 * (p - 2) / (p + 2)
    H = 0.0
    v = 0.0
    for _ in range(200):
        H = math.sqrt(fmp * fmp / 3.0 * (0.5 * v * v + 1.0 / p))
        v = 1.0 / (3.0 * H)
    c = 1.0 / math.sqrt(2.0)
    return {"p": p, "alpha": alpha, "fstar_over_mp": fmp, "omega_over_fstar": om, "gauge_e": e, "qA": qA,
            "phi0": (c, c), "dphi0": (-v * c, -v * c), "H0": H}


def accuracy_measurement(args, stream):
    """Friedmann-constraint error Delta_e (sections 8.2 and 8.3, accuracy tests)
    of the chosen integrators on the p = 4 working examples at k_IR = 0.6,
    dt = 0.01, FP64, from one vacuum-fluctuation start: the U(1)-charged
    inflaton (q_A* = 100), or the SU(2) x U(1) doublet with a singlet
    (q_A* = q_B* = q* = 100).  Sampled at the start and every 5 program-time
    units, with the device time of each run and the energy fractions of the
    sectors."""
    import torch

    import paper_2006_15122_gb300 as cl

    st = u1_inflaton_setup()
    N, kIR, dt = args.acc_N, 0.6, 0.01
    nsteps = int(round(args.acc_eta / dt))
    every = int(round(5.0 / dt))
    su2 = args.acc_model == "su2u1"
    if su2:
        # the doublet's stored components: |Phi|^2 = 1/2 (canonical norm 1) split evenly, radial velocity
        c = 1.0 / math.sqrt(8.0)
        v = st["dphi0"][0] * math.sqrt(2.0)  # the radial canonical speed
        st = dict(st, phi0=(c, c, c, c), dphi0=(v * c, v * c, v * c, v * c), qB=st["qA"], q=st["qA"],
                  gauge_e_su2=2.0 * math.sqrt(st["qA"]) * st["omega_over_fstar"])
        name = "SU(2) x U(1) doublet + singlet, V = (1/p)(2|Phi|^2)^(p/2) + q |Phi|^2 chi^2"
    else:
        name = "U(1) charged inflaton, V = (1/p)(2|phi|^2)^(p/2)"
    out = {"model": name, "setup": st, "N": N, "kIR": kIR, "dt": dt, "eta_end": nsteps * dt, "precision": "f64",
           "runs": {}}
    for integ in args.acc_integrators.split(","):
        if su2:
            model = cl.make_model(kind=cl.CL_MODEL_SU2, n_fields=2, alpha=st["alpha"],
                                  fstar_over_mp=st["fstar_over_mp"], omega_over_fstar=st["omega_over_fstar"], lam=1.0,
                                  q=st["q"], gauge_e=st["gauge_e_su2"], gauge_e_u1=st["gauge_e"],
                                  potential=cl.CL_POT_MONOMIAL, pexp=st["p"])
        else:
            model = cl.make_model(kind=cl.CL_MODEL_U1, alpha=st["alpha"], fstar_over_mp=st["fstar_over_mp"],
                                  omega_over_fstar=st["omega_over_fstar"], lam=1.0, gauge_e=st["gauge_e"],
                                  potential=cl.CL_POT_MONOMIAL, pexp=st["p"])
        lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, integ, cl.CL_FP64), cl.make_init(
            phi0=st["phi0"], dphi0=st["dphi0"], seed=1, spectrum=1), stream=stream)
        t, de, dg, a, frac = [], [], [], [], []

        def sample():
            mm = lat.measure_means()
            t.append(mm["t"])
            de.append(mm["hubble_violation"])
            dg.append(mm["gauss_violation"])
            a.append(mm["a"])
            r = mm["rho"]
            if su2:
                frac.append({"inflaton": (mm["EK"][0] + mm["EG"][0] + mm["EV"][0]) / r,
                             "su2": (mm["EK"][1] + mm["EG"][1]) / r, "u1": (mm["EK"][2] + mm["EG"][2]) / r,
                             "chi": (mm["EK"][3] + mm["EG"][3]) / r})
            else:
                frac.append({"inflaton": (mm["EK"][0] + mm["EG"][0] + mm["EV"][0]) / r,
                             "u1": (mm["EK"][1] + mm["EG"][1]) / r})

        sample()
        ms = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            e0.record(stream)
            lat.evolve(k)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            done += k
            sample()
        lat.close()
        out["runs"][integ] = {"t": t, "delta_e": de, "gauss_violation": dg, "a": a, "energy_fractions": frac,
                              "device_ms": ms, "ms_per_step": ms / nsteps, "delta_e_end": de[-1],
                              "delta_e_max": max(de)}
    return out


def fp64_error_measurement(lat32, N, steps, seed, stream):
    """The FP32 run's error against the same lattice in FP64 (section 4.3.2's
    scheme with FP64 arrays, same seed, same number of steps): max-norm relative
    error of each fluctuation array, relative errors of the means, a and b, and
    of the phi and chi spectra (largest over the shells); plus the FP64 rate."""
    import torch

    import paper_2006_15122_gb300 as cl

    model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, fstar_over_mp=FSTAR_MP, omega_over_fstar=OMEGA_FSTAR,
                          lam=1.0, q=QSTAR)
    lat64 = cl.Lattice(model, cl.make_grid(N, KIR, DT, "vv4", cl.CL_FP64), cl.make_init(phi0=(1.0, 0.0), seed=seed),
                       stream=stream)
    lat64.evolve(1)  # records the one-step graph; the timed call below records its own
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat64.evolve(steps - 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    out = {"steps": steps, "fp64_site_updates_per_s": N ** 3 * (steps - 1) / (ms64 / 1e3),
           "fp64_ms_per_step": ms64 / (steps - 1), "fluct_maxnorm_rel": {}, "mean_rel": {}}
    m32, m64 = lat32.measure_means(), lat64.measure_means()
    names = {cl.FIELD(0): "phi", cl.FIELD(1): "chi", cl.MOMENTUM(0): "pi_phi", cl.MOMENTUM(1): "pi_chi"}
    x = torch.empty((N, N, N), device="cuda", dtype=torch.float64)
    y = torch.empty((N, N, N), device="cuda", dtype=torch.float64)
    for w, nm in names.items():
        lat32.get_field(w, x)
        lat64.get_field(w, y)
        mx, my = x.mean().item(), y.mean().item()
        dy = (y - my)
        scale = dy.abs().max().item()
        out["fluct_maxnorm_rel"][nm] = ((x - mx) - dy).abs().max().item() / scale
        ref = abs(my) if nm == "phi" else dy.pow(2).mean().sqrt().item()  # zero-mean fields: against their rms
        out["mean_rel"][nm] = abs(mx - my) / ref
    del x, y
    out["a_rel"] = abs(m32["a"] - m64["a"]) / m64["a"]
    out["b_rel"] = abs(m32["b"] - m64["b"]) / abs(m64["b"])
    out["energy_rel"] = {k: max(abs(m32[k][i] - m64[k][i]) / abs(m64[k][i]) for i in range(2)) for k in ("EK", "EG", "EV")}
    out["spectrum_max_rel"] = {}
    for f, nm in ((0, "phi"), (1, "chi")):
        _, D32, _ = lat32.spectrum(f, 0)
        _, D64, c = lat64.spectrum(f, 0)
        sel = (c > 0) & (D64 > 0)
        sel[0] = False
        out["spectrum_max_rel"][nm] = float(max(abs(D32[sel] - D64[sel]) / D64[sel]))
    lat64.close()
    torch.cuda.empty_cache()
    return out


def replica_seed(rank):
    """Under torchrun every rank evolves its own replica, drawn from seed = rank."""
    return rank


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (all ranks start together after a barrier)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(sites, steps, world, ms):
    """Site updates per second of all replicas together over the max-over-ranks time."""
    return world * sites * steps / (ms / 1e3)


def surrogate_measurement(args, stream):
    """Training and query time of the surrogate network (2-256-256-256-34) on
    synthetic data of the scan's shape: 32768 rows of (log10 q, t) -> 34 smooth
    observables, batch 512, args.surrogate_epochs epochs, Adam with a cosine step size."""
    import numpy as np
    import torch

    import paper_2006_15122_gb300 as cl

    rng = np.random.default_rng(0)
    n = 32768
    X = np.stack([rng.uniform(2, 5, n), rng.uniform(0, 200, n)], axis=1).astype(np.float32)
    k = np.linspace(0.5, 2.0, 32)
    Y = np.concatenate([np.tanh(X[:, 1:] / 50.0 - X[:, :1] / 2.0), np.cos(X[:, 1:] / 30.0) * np.sin(X[:, :1]),
                        np.log1p(np.abs(np.outer(X[:, 0], k) - X[:, 1:] / 60.0))], axis=1).astype(np.float32)
    net = cl.Surrogate(2, 34, 256, 3, seed=0, stream=stream)
    net.train(X[:1024], Y[:1024], epochs=2, batch=512)  # records the epoch graph of a small set
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = net.train(X, Y, epochs=args.surrogate_epochs, batch=512, lr=2e-3, lr_end=2e-5, shuffle=True)
    t_train = time.perf_counter() - t0
    net.predict(X[:4096])
    t0 = time.perf_counter()
    net.predict(X[:4096])
    t_query = time.perf_counter() - t0
    net.close()
    steps = args.surrogate_epochs * (n // 512)
    return {"metric": "surrogate training time", "value": t_train, "unit": "s", "higher_is_better": False,
            "config": {"workload": "MLP 2-256-256-256-34 GELU on 32768 synthetic rows shaped like the scan's "
                                   "training set, batch 512, %d epochs" % args.surrogate_epochs},
            "us_per_minibatch": 1e6 * t_train / steps, "loss_first_last": [float(hist[0]), float(hist[-1])],
            "query_4096_rows_ms": 1e3 * t_query}


def run_scan(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    line = scan_measurement(args, torch.cuda.current_stream(), dist)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.scan:
        return run_scan(args)
    if args.gauge_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        N = args.gauge_N or (256 if args.gauge_only == "u1" else 128)
        print(json.dumps(gauge_measurement(args.gauge_only, N, args.gauge_steps, torch.cuda.current_stream())),
              flush=True)
        return
    if args.surrogate:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(surrogate_measurement(args, torch.cuda.current_stream())), flush=True)
        return
    if args.accuracy:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(accuracy_measurement(args, torch.cuda.current_stream())), flush=True)
        return
    import torch

    import paper_2006_15122_gb300 as cl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    N = args.N
    stream = torch.cuda.current_stream()
    model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, fstar_over_mp=FSTAR_MP, omega_over_fstar=OMEGA_FSTAR,
                          lam=1.0, q=QSTAR)
    grid = cl.make_grid(N, KIR, DT, "vv4", cl.CL_FP32)
    lat = cl.Lattice(model, grid, cl.make_init(phi0=(1.0, 0.0), seed=replica_seed(rank)), stream=stream)

    for _ in range(args.warmup):
        lat.evolve(1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.evolve(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, "cuda")
    mm = lat.measure_means()
    npass = 3 * args.steps + 1
    value = whole_job_rate(N ** 3, args.steps, world, ms)
    peak, peak_kind = measured_peaks()
    alg_bytes = BYTES_PER_SITE_PASS * N ** 3
    achieved = alg_bytes / (ms / 1e3 / npass) / 1e9

    err64 = None
    if not args.no_fp64:
        try:
            err64 = fp64_error_measurement(lat, N, args.warmup + args.steps, replica_seed(rank), stream)
        except Exception as exc:  # the FP32 number above stands on its own
            err64 = {"error_running": repr(exc)}
    e2e = None
    if not args.no_e2e:
        # end to end through the public API with pinned host buffers: every step
        # uploads the stored state (four FP32 fluctuation arrays and their FP64
        # means, lattice_set_stored), advances one step, reads the means back
        which = [cl.FIELD(0), cl.FIELD(1), cl.MOMENTUM(0), cl.MOMENTUM(1)]
        host = [torch.empty((N, N, N), dtype=torch.float32, pin_memory=True) for _ in range(4)]
        means = [lat.get_stored(w, host[i])[1] for i, w in enumerate(which)]
        mm0 = lat.measure_means()
        reps = 8  # about 1 s: an occasional slow upload (0.33 s instead of 0.08 s) is averaged over more steps
        ph = {"set_stored": 0.0, "evolve": 0.0, "measure": 0.0}
        uploads = []
        for i, w in enumerate(which):  # one untimed pass over the host buffers
            lat.set_stored(w, host[i], means[i])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            ta = time.perf_counter()
            for i, w in enumerate(which):
                lat.set_stored(w, host[i], means[i])
            tb = time.perf_counter()
            lat.set_background(mm0["a"], mm0["b"], mm0["t"])
            lat.evolve(1)
            lat.measure_means()  # synchronizes: the step is done when it returns
            tc = time.perf_counter()
            ph["set_stored"] += tb - ta
            ph["evolve"] += tc - tb
            uploads.append(1e3 * (tb - ta))
        t1 = time.perf_counter()
        e2e = {"value": world * N ** 3 * reps / (t1 - t0), "unit": "site-updates/s",
               "h2d_bytes_per_step": 4 * 4 * N ** 3 + 4 * 8, "d2h_bytes_per_step": 320,
               "note": "per step: the 4 FP32 fluctuation arrays and their FP64 means H2D from pinned memory via "
                       "lattice_set_stored, one VV4 step, lattice_measure_means D2H",
               "ms_per_step_phases": {"upload": 1e3 * ph["set_stored"] / reps,
                                      "step_and_measure": 1e3 * ph["evolve"] / reps},
               "h2d_GBs": 4 * 4 * N ** 3 / (ph["set_stored"] / reps) / 1e9, "upload_ms_per_rep": uploads}
        del host
    lat.close()
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(128)
    gauge = None
    if rank == 0 and not args.no_gauge:
        try:
            gauge = {"u1": gauge_measurement("u1", 256, 20, stream), "su2": gauge_measurement("su2", 128, 10, stream),
                     "su2u1": gauge_measurement("su2u1", 128, 10, stream)}
        except Exception as exc:
            gauge = {"error_running": repr(exc)}
    ens = None
    if rank == 0 and args.with_scan:
        try:
            ens = scan_measurement(args, stream)
        except Exception as exc:  # the lattice number above stands on its own
            ens = {"error_running": repr(exc)}
    if rank == 0:
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(N), parallelism="replicas" if world > 1 else "single"),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": measured_traffic(N), "peak_kind": peak_kind,
                         "kernel": "scalar_pass_kernel<float,2,2,16>", "bytes_per_launch": alg_bytes,
                         "launch_ms": ms / npass},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": npass, "clocks": clk,
            "hubble_violation": mm["hubble_violation"], "a": mm["a"], "error_vs_fp64": err64,
            "ensemble_scan": ens, "gauge_passes": gauge,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
