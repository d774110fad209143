"""Benchmark: eigenpairs/s of POLFED on synthetic disordered chains (one GB300 per rank).

The work is a stream of back-to-back polfed_eigs runs on fresh disorder
realizations (spectral bounds, K from the density of states, block Lanczos on
the Chebyshev filter with full re-orthogonalization, Ritz vectors,
Rayleigh-Ritz with H~, refinement sweeps, residual check).  A *step* is one
block-Lanczos step of that stream (one Chebyshev filter of the n_b block,
re-orthogonalization, QR and, from some step on, the T_j eigenproblem with
the convergence test), or one refinement sweep; the library reports every
step boundary through its progress hook.  --warmup W steps are untimed, then
exactly --steps K steps are timed (barrier + device synchronize on both
sides), and the run in progress at the end is finished untimed so that its
pairs are verified.  Each run's verified pairs are credited to the timed
region in proportion to the share of the run's time that lies inside it.
Ranks (torchrun) run independent realizations (weak scaling, no data-path
collective).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --filter-only [--workload ...] [--precision f32|df64|f64] [--K 6]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import polfed_inputs as I  # noqa: E402

METRIC = "eigenpairs/s at L=22, ε=0.5 (resid≤1e-8‖H‖); filter GB/s vs HBM peak"
WORKLOADS = {
    # name: (builder, L, W, N_ev, n_b, config id of the field generator)
    "L22_xxz_W3": (I.xxz, 22, 3.0, 500, 64, 4),
    "L20_j1j2_W4": (I.j1j2, 20, 4.0, 200, 32, 2),
    "L14_xxz_W3": (I.xxz, 14, 3.0, 50, 16, 1),
    "L24_j1j2_W5": (I.j1j2, 24, 5.0, 1000, 64, 5),
    # free-fermion point (Delta = 0, J2 = 0, open chain): exact spectrum at any L
    "L22_ff_W3": (I.free_fermion, 22, 3.0, 500, 64, 6),
    "L24_ff_W3": (I.free_fermion, 24, 3.0, 1000, 64, 6),
}
# 64 XXZ rings, L = 16 / 18 alternating, W cycling {1,2,3,4,6,8}, N_ev cycling {50,100,200}
BATCHED = {"batched64_L16_L18": (64, (16, 18), (1.0, 2.0, 3.0, 4.0, 6.0, 8.0), (50, 100, 200), 3),
           # a small batch of the same kind for quick checks
           "batched8_L12_L14": (8, (12, 14), (1.0, 3.0, 6.0, 8.0), (20, 40), 3)}
PREC = {"df64": 2, "f64": 0, "f32": 1}
DOS = {"moments": 0, "gamma": 1, "kpm": 2, "mlp": 3}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def tma_kernel_source_sha():
    """sha256 (16 hex) of the TMA step kernel's source text (from its section
    comment to the slice-conversion code that follows it)."""
    src = open(os.path.join(ROOT, "paper_2005_09534_gb300", "csrc", "hamiltonian.cu")).read()
    a = src.index("// ------------------------------------------------- TMA-pipelined step kernel")
    b = src.index("template <class NT>\nstruct Conv;")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def step_kernel_traffic(precision, workload):
    """DRAM traffic of one step-kernel launch from the committed ncu summary of
    this workload and precision, if it was taken on the current kernel source
    (else None)."""
    try:
        sha = tma_kernel_source_sha()
        with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")) as f:
            d = json.load(f)
        e = d.get(f"{workload}:{precision}")
        if e and e.get("source_sha") == sha:
            return {"dram_bytes_per_launch_scaled": e["dram_bytes_per_launch"], "source": e.get("summary")}
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle legs
def host_threads():
    """Host cores this process may use (the affinity mask, else the CPU count)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_dense_sample(seconds=12.0):
    """The CPU oracle (dense ED of the S^z=0 block, LAPACK eigh) on L=14 XXZ chains,
    N_ev=50 nearest eps=0.5, repeated over realizations for about `seconds`."""
    import oracle as O
    t0 = time.perf_counter()
    n_pairs, n_real = 0, 0
    while True:
        m = I.xxz(14, 3.0, 1, 100 + n_real)
        r = O.eigs_nearest(m.L, m.J1, m.J2, m.Delta, m.h, True, 0.5, 50)
        n_pairs += len(r["evals"])
        n_real += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": n_pairs / dt, "unit": "eigenpairs/s", "cores": host_threads(), "kind": "oracle",
            "sample": f"dense ED (numpy eigh, default BLAS threads) of {n_real} L=14 XXZ W=3 realizations, "
                      f"N_ev=50 each, {dt:.1f} s"}


def _column_worker(conn, workload, realization, chunk, ncols):
    """A host process that owns one column chunk of the workload's block and runs
    the oracle's filter on it when asked (n Chebyshev steps per request)."""
    import oracle as O
    builder, L, W, n_ev, n_b, cfg = WORKLOADS[workload]
    md = builder(L, W, cfg, realization)
    H, _ = O.sparse_hamiltonian(md.L, md.J1, md.J2, md.Delta, md.h, md.periodic)
    Ht = (H / field_free_bound(md)).tocsr()  # H~ for [e_lo, e_hi] = [-bound, bound] (bound >= ||H||)
    X = I.block(H.shape[0], ncols, 11 + chunk)
    conn.send("ready")
    while True:
        n = conn.recv()
        if n is None:
            break
        c, D = O.cheb_coeffs(0.0, n)
        t0 = time.perf_counter()
        O.filter_matrix_powers(Ht, X, c, D)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OracleFilter:
    """The oracle's Chebyshev filter (filter_matrix_powers: the matrix three-term
    recurrence on a scipy CSR H~) on one realization of a workload, its n_b
    columns split over `procs` host processes (spawned), one column chunk per
    process (the paper's column-per-core parallelism, Supplement "Technical
    details")."""

    def __init__(self, workload, procs, realization=0):
        import multiprocessing as mp
        builder, L, W, n_ev, n_b, cfg = WORKLOADS[workload]
        self.workload, self.n_ev, self.n_b, self.L = workload, n_ev, n_b, L
        self.realization = realization
        self.dim = math.comb(L, L // 2)
        self.threads = max(1, min(procs, n_b))
        sizes = [len(c) for c in np.array_split(np.arange(n_b), self.threads)]
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        self.conns, self.procs = [], []
        for k, nc in enumerate(sizes):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_column_worker, args=(b, workload, realization, k, nc), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for a in self.conns:
            assert a.recv() == "ready"
        self.t_build = time.perf_counter() - t0

    def steps(self, n):
        """n Chebyshev steps of the whole block (all chunks in parallel); returns the seconds taken."""
        t0 = time.perf_counter()
        for a in self.conns:
            a.send(n)
        for a in self.conns:
            a.recv()
        return time.perf_counter() - t0

    def rate(self, seconds, n=4):
        """Seconds per Chebyshev step of the block, measured for about `seconds`."""
        self.steps(n)  # warm-up
        done, t = 0, 0.0
        while t < seconds:
            t += self.steps(n)
            done += n
        return t / done, done, t

    def method_order(self, n_ev):
        """K and block steps of a plain FP64 POLFED run of this realization, from
        the oracle: bounds (ARPACK), exact sector moments, the Gaussian density at
        the middle of the spectrum and the order rule for (1 + 0.2) N_ev
        accessible values; block steps at the Supplement's convergence onset
        m s = 2 N_ev (Fig. S1), the fewest any run needs."""
        import oracle as O
        builder, L, W, _, n_b, cfg = WORKLOADS[self.workload]
        md = builder(L, W, cfg, self.realization)
        H, _ = O.sparse_hamiltonian(md.L, md.J1, md.J2, md.Delta, md.h, md.periodic)
        lo, hi = O.extreme_eigenvalues(H)
        mean, var = O.sector_moments(H)
        rho_t = O.gaussian_rho(self.dim, mean, var, 0.5 * (lo + hi)) * 0.5 * (hi - lo)
        K = O.order_for_window(rho_t, 1.2 * n_ev)
        m = int(math.ceil(2.0 * n_ev / self.n_b))
        return K, m

    def close(self):
        for a in self.conns:
            try:
                a.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)


def oracle_baseline(workload, K_run, m_run, km_source, seconds=12.0):
    """cpu_baseline of the GPU line: the oracle's filter on the workload, all host
    threads, timed for about `seconds`; the eigenpairs/s figure extrapolates the
    measured seconds per Chebyshev block step to K x m block steps (refinement,
    re-orthogonalization and the other FP64 work are left out, so it is an
    upper bound on the CPU rate)."""
    f = OracleFilter(workload, host_threads())
    try:
        t_step, n, t = f.rate(seconds)
    finally:
        f.close()
    run_s = K_run * m_run * t_step
    return {"value": f.n_ev / run_s, "unit": "eigenpairs/s", "cores": f.threads, "kind": "oracle",
            "sample": f"oracle filter_matrix_powers on the {workload} sparse H~ (dim {f.dim}, {f.n_b} columns "
                      f"over {f.threads} processes, scipy CSR SpMM): {n} Chebyshev block steps in {t:.1f} s measured "
                      f"({t_step:.4f} s per step); eigenpairs/s = N_ev / (K x m x that), K x m = {K_run} x {m_run} "
                      f"({km_source}); refinement and FP64 dense work left out",
            "seconds_per_cheb_step": t_step, "cheb_steps_timed": n, "seconds_timed": t,
            "extrapolated_run_s": run_s}


def oracle_batched_sample(ms, nev, sts, seconds=5.0):
    """The batched workload on the host: the oracle's filter rate per Chebyshev step for one
    realization of each chain length (n_b = 16, one column chunk per thread), extrapolated by
    every realization's own K x m x (n_b / 16) block steps from the GPU run."""
    import oracle as O
    rate = {}
    thr = host_threads()
    pool = ThreadPoolExecutor(max_workers=min(thr, 16))
    for md in ms:
        if md.L in rate:
            continue
        H, _ = O.sparse_hamiltonian(md.L, md.J1, md.J2, md.Delta, md.h, md.periodic)
        bound = 2 * md.L * (0.5 + abs(md.Delta) / 4) + 0.5 * float(np.abs(md.h).sum())
        Ht = (H / bound).tocsr()
        X = I.block(H.shape[0], 16, 12)
        chunks = [np.ascontiguousarray(X[:, c]) for c in np.array_split(np.arange(16), min(thr, 16))]
        c, D = O.cheb_coeffs(0.0, 4)
        steps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            list(pool.map(lambda x: O.filter_matrix_powers(Ht, x, c, D), chunks))
            steps += 4
        rate[md.L] = (time.perf_counter() - t0) / steps
    pool.shutdown()
    t_run = sum(st["K"] * st["m"] * max(1, st["n_b"] // 16) * rate[md.L] for md, st in zip(ms, sts))
    return {"value": sum(nev) / t_run, "unit": "eigenpairs/s", "cores": min(thr, 16), "kind": "oracle",
            "sample": "oracle filter_matrix_powers on one sparse H~ per chain length (16 columns over "
                      f"{min(thr, 16)} threads, scipy CSR): "
                      + ", ".join(f"L={L}: {t:.4f} s/step" for L, t in sorted(rate.items()))
                      + f"; extrapolated by each realization's K x m block steps: {t_run:.0f} s for the batch "
                        "(refinement and FP64 work left out)",
            "extrapolated_run_s": t_run}


def run_reference(args):
    """--impl reference: the CPU oracle on the host cores.  Each step is a bounded
    sample of the workload: `cheb_per_step` Chebyshev steps of the n_b block
    through the oracle's filter, one column chunk per thread.  The eigenpairs/s
    value extrapolates the measured seconds per Chebyshev step to the K x m
    block steps the oracle's own order rule and the Supplement's convergence
    onset give for this realization."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in BATCHED:
        wl = "L14_xxz_W3"
    else:
        wl = args.workload
    builder, L, W, n_ev, n_b, c_id = WORKLOADS[wl]
    f = OracleFilter(wl, host_threads())
    t_setup0 = time.perf_counter()
    K, m = f.method_order(n_ev)
    t_setup = time.perf_counter() - t_setup0
    n_cheb = 8 if f.dim > 100000 else 64
    for _ in range(args.warmup):
        f.steps(n_cheb)
    per = []
    for _ in range(args.steps):
        per.append(f.steps(n_cheb))
    f.close()
    t_timed = float(sum(per))
    t_step = t_timed / (n_cheb * args.steps)
    run_s = K * m * t_step
    value = n_ev / run_s
    cfg = {"workload": wl, "L": L, "W": W, "N_ev": n_ev, "n_b": n_b, "eps": 0.5, "dim": f.dim,
           "step": f"{n_cheb} Chebyshev steps of the {n_b}-column block (oracle filter, {f.threads} processes)",
           "K": K, "m": m,
           "K_m_source": "oracle: ARPACK bounds, exact sector moments, Gaussian density, order rule for 1.2 N_ev; "
                         "m s = 2 N_ev (convergence onset of the Supplement)"}
    if args.workload in BATCHED:
        cfg["stand_in_for"] = args.workload
    cb = {"value": value, "unit": "eigenpairs/s", "cores": f.threads, "kind": "oracle",
          "sample": f"{args.steps} timed steps of {n_cheb} Chebyshev block steps each on {wl} (dim {f.dim}): "
                    f"{t_step:.4f} s per Chebyshev step measured; eigenpairs/s extrapolated by K x m = {K} x {m}",
          "seconds_per_cheb_step": t_step, "extrapolated_run_s": run_s, "setup_s": round(t_setup + f.t_build, 2)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_timed / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
class StepWindow:
    """Counts step boundaries reported by the library's progress hook and takes
    the timed region: after `warmup` boundaries it synchronizes, passes a
    barrier and records a CUDA event on the context's stream, the wall clock and
    the library's counters; after `warmup + steps` boundaries it does the same
    to close the region."""

    def __init__(self, torch, pf, stream, warmup, steps, dist, clocks):
        self.torch, self.pf, self.stream = torch, pf, stream
        self.W, self.K = warmup, steps
        self.dist, self.clocks = dist, clocks
        self.n = 0
        self.ev = {"ref": self.event(), "start": None, "stop": None}
        self.ev["ref"].record(stream)
        self.wall = {}
        self.cnt = {}

    def event(self):
        return self.torch.cuda.Event(enable_timing=True)

    def ms(self, e):
        """Offset of event e from the reference event, ms (same stream: a common timeline)."""
        return self.ev["ref"].elapsed_time(e)

    @property
    def started(self):
        return self.ev["start"] is not None

    @property
    def done(self):
        return self.ev["stop"] is not None

    def hook(self, phase, index):
        if phase not in (self.pf.PHASE_BLOCK, self.pf.PHASE_REFINE):
            return
        self.n += 1
        if self.n == self.W:
            self.open()
        elif self.n == self.W + self.K:
            self.close()

    def open(self):
        self.torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        if self.clocks:
            self.clocks.start()
        self.cnt["start"] = self.pf.get_counters()
        self.wall["start"] = time.perf_counter()
        e = self.event()
        e.record(self.stream)
        self.ev["start"] = e

    def close(self):
        e = self.event()
        e.record(self.stream)
        self.torch.cuda.synchronize()
        self.wall["stop"] = time.perf_counter()
        self.cnt["stop"] = self.pf.get_counters()
        self.ev["stop"] = e
        if self.dist:
            self.dist.barrier()


def overlap(a0, a1, b0, b1):
    return max(0.0, min(a1, b1) - max(a0, b0))


def credited_pairs(spans, w0, w1):
    """Eigenpairs credited to the timed region [w0, w1]: each run (start, end,
    verified pairs) contributes its pairs times the share of its span inside
    the region."""
    return sum(ok * overlap(s, e, w0, w1) / max(e - s, 1e-12) for s, e, ok in spans)


def run_single(args, pf, torch, dev, world, rank, local, dist):
    builder, L, W, n_ev, n_b, cfg = WORKLOADS[args.workload]
    dim = pf.basis_build(L, L // 2)
    stream = torch.cuda.Stream(device=dev)
    ctx = pf.Ctx(local)
    ctx.set_stream(stream)
    opts = pf.opts_default()
    opts.precision = PREC[args.precision]
    opts.dos_rule = DOS[args.dos]
    net, mlp_info = None, None
    if args.dos == "mlp":
        net, mlp_info = train_predictor(pf, ctx, builder, L, W, cfg)
    evecs = torch.empty((n_ev, dim), dtype=torch.float64, device=dev)  # column-major dim x N_ev
    host_evecs = torch.empty((n_ev, dim), dtype=torch.float64, pin_memory=True)
    fields_pinned = torch.empty(L, dtype=torch.float64, pin_memory=True)
    clocks = Clocks(local) if rank == 0 else None
    win = StepWindow(torch, pf, stream, args.warmup, args.steps, dist, clocks)
    ctx.set_progress(win.hook)
    torch.cuda.synchronize()
    if win.W == 0:
        win.open()
    runs = []
    r = 0
    while not win.done:
        m = builder(L, W, cfg, timed_realization(r, world, rank))
        e_s, e_e = win.event(), win.event()
        t_s = time.perf_counter()
        e_s.record(stream)
        fields_pinned.copy_(torch.from_numpy(m.h))
        model = pf.Model(L, m.J1, m.J2, m.Delta, fields_pinned.numpy(), m.periodic)
        if net is not None:  # the learned predictor sets K (inference inside the run)
            emin, emax, rho = net.predict(model, W)
            opts.rho_hint = rho
            # its bounds are not passed: the Lanczos probe runs anyway (the target needs exact extremes),
            # and the probe's interval is both tighter and centred on the target (sigma = 0 exactly, so
            # the odd Chebyshev terms vanish and half of the filter steps skip reading X)
            opts.emin_hint, opts.emax_hint = 0.0, 0.0
        ev, res, st, rc = pf.eigs(ctx, model, 0.5, n_ev, 0, n_b, opts, d_evecs=evecs, allow_noconv=True)
        e_e.record(stream)
        with torch.cuda.stream(stream):
            host_evecs.copy_(evecs, non_blocking=True)
        stream.synchronize()
        t_e = time.perf_counter()
        hn = max(abs(st["E_min"]), abs(st["E_max"]))
        ok = int(np.sum(res[: len(ev)] <= 1e-8 * hn)) if rc == 0 else 0
        runs.append({"realization": timed_realization(r, world, rank), "ev_s": e_s, "ev_e": e_e, "t_s": t_s,
                     "t_e": t_e, "ok": ok, "rc": rc, "st": st, "max_rel_resid": float(np.max(res) / hn),
                     "evals": ev})
        r += 1
    ctx.set_progress(None)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    # timed region on the device timeline and on the wall clock
    w0, w1 = win.ms(win.ev["start"]), win.ms(win.ev["stop"])
    t_dev = (w1 - w0) / 1e3
    t_wall = win.wall["stop"] - win.wall["start"]
    h2d, d2h, in_window = 0, 0, []
    for run in runs:
        run["s"], run["e"] = win.ms(run["ev_s"]), win.ms(run["ev_e"])
    pairs_dev = credited_pairs([(x["s"], x["e"], x["ok"]) for x in runs], w0, w1)
    pairs_wall = credited_pairs([(x["t_s"], x["t_e"], x["ok"]) for x in runs], win.wall["start"], win.wall["stop"])
    for run in runs:
        s, e = run["s"], run["e"]
        od = overlap(s, e, w0, w1)
        ow = overlap(run["t_s"], run["t_e"], win.wall["start"], win.wall["stop"])
        if od > 0 or ow > 0:
            in_window.append(run)
        # a run's copies (fields in, eigenvectors and values out) are credited like its pairs
        share_w = ow / max(run["t_e"] - run["t_s"], 1e-12)
        h2d += L * 8 * share_w
        d2h += (n_ev * dim * 8 + 2 * n_ev * 8) * share_w
        run["dev_s"] = (e - s) / 1e3
        run["wall_s"] = run["t_e"] - run["t_s"]
        run["share_in_window"] = od / max(e - s, 1e-9)
    t_dev, t_wall, pairs_all, pairs_wall_all = reduce_ranks(torch, dev, dist, t_dev, t_wall, pairs_dev, pairs_wall)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    c0, c1 = win.cnt["start"], win.cnt["stop"]
    peak, peak_kind = peaks()
    names = {0: "f64", 1: "f32", 2: "df64"}
    kinds = {}
    for k in range(3):
        n = c1["kind_launches"][k] - c0["kind_launches"][k]
        g = c1["kind_gpu_s"][k] - c0["kind_gpu_s"][k]
        b = c1["kind_alg_bytes"][k] - c0["kind_alg_bytes"][k]
        if n > 0 and g > 0:
            kinds[names[k]] = {"launches": int(n), "avg_launch_us": round(1e6 * g / n, 2),
                               "alg_bytes_per_launch": b / n, "achieved_gbs": round(b / g / 1e9, 1),
                               "share_of_step": round(g / max(t_dev, 1e-12), 4)}
    dom = max(kinds, key=lambda k: kinds[k]["share_of_step"]) if kinds else args.precision
    d = kinds.get(dom, {"achieved_gbs": 0.0, "alg_bytes_per_launch": 0.0, "avg_launch_us": 0.0, "launches": 0,
                        "share_of_step": 0.0})
    tr = step_kernel_traffic(dom, args.workload)
    roof = {"bound": "hbm", "achieved": d["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": round(d["achieved_gbs"] / peak, 4),
            "traffic": (tr or {}).get("dram_bytes_per_launch_scaled"),
            "peak_kind": f"of {peak_kind}",
            "kernel": f"k_ham_step_tma<{dom}> (Clenshaw step on a 128-byte column slice)",
            "alg_bytes_per_launch": d["alg_bytes_per_launch"], "avg_launch_us": d["avg_launch_us"],
            "launches": d["launches"], "share_of_step": d["share_of_step"], "by_kind": kinds}
    if tr:
        roof["traffic_source"] = tr.get("source")
    value = pairs_all / t_dev
    line = {"metric": METRIC, "value": round(value, 4), "unit": "eigenpairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_dev / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": args.workload, "L": L, "dim": dim, "hamiltonian": builder.__name__,
                       "W": W, "N_ev": n_ev, "n_b": n_b, "eps": 0.5, "dos_rule": args.dos,
                       "step": "one block-Lanczos step or refinement sweep of back-to-back polfed_eigs runs",
                       "pairs_credited": round(pairs_all, 2),
                       "runs": [{"realization": x["realization"], "K": x["st"]["K"], "m": x["st"]["m"],
                                 "refine": x["st"]["n_refine"], "restarts": x["st"]["n_restarts"],
                                 "fallback_df64": x["st"]["fallback_df64"], "status": x["rc"],
                                 "verified_pairs": x["ok"], "max_resid_over_normH": x["max_rel_resid"],
                                 "dev_s": round(x["dev_s"], 3), "wall_s": round(x["wall_s"], 3),
                                 "share_in_window": round(x["share_in_window"], 4),
                                 "phase_s": {k[2:]: round(x["st"][k], 2) for k in
                                             ("t_bounds", "t_filter", "t_reorth", "t_qr", "t_teig", "t_ritz",
                                              "t_total")}}
                                for x in runs],
                       "parallelism": f"replicas x{world}",
                       "l2": "per-step working set (>= 3 x 90 MB slices + 10 GB Lanczos basis) >> L2, no flush"},
            "roofline": roof,
            "e2e": {"value": round(pairs_wall_all / t_wall, 4), "unit": "eigenpairs/s",
                    "h2d_bytes_per_step": int(round(h2d / args.steps)),
                    "d2h_bytes_per_step": int(round(d2h / args.steps)),
                    "copies": "each run copies its fields from pinned host memory and its N_ev eigenvectors "
                              "and values back to pinned memory; bytes credited by the run's share of the "
                              "timed region, like its pairs"},
            "gpu_launches": int(c1["launches"] - c0["launches"]),
            "clocks": ck}
    if mlp_info:
        line["config"]["mlp"] = mlp_info
    if world == 1 and not args.no_cpu_baseline:
        Ks = [x["st"]["K"] for x in in_window] or [runs[-1]["st"]["K"]]
        ms_ = [x["st"]["m"] for x in in_window] or [runs[-1]["st"]["m"]]
        line["cpu_baseline"] = oracle_baseline(args.workload, int(round(np.mean(Ks))), int(round(np.mean(ms_))),
                                               "mean K and m of the timed GPU runs")
        if L > 14:
            line["cpu_dense_ed_L14"] = oracle_dense_sample(8.0)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_filter_only(args, pf, torch, dev):
    """One polfed_cheb_filter call (sigma = 0, order --K) on a seeded block of the
    workload's Hamiltonian, for kernel profiling (ncu): K + 1 step-kernel launches
    per 128-byte column slice.  Batched workloads: one polfed_cheb_filter_batched
    call over their realizations (n_b = 16)."""
    kind = PREC[args.precision]
    dt = torch.float32 if kind == pf.F32 else torch.float64
    if args.workload in BATCHED:
        n, Ls, Wc, Nc, cfg = BATCHED[args.workload]
        ms, Xs, Ys = [], [], []
        for r in range(n):
            m = I.xxz(Ls[r % len(Ls)], Wc[r % len(Wc)], cfg, r)
            d = pf.basis_build(m.L, m.L // 2)
            ms.append(m)
            Xs.append(torch.from_numpy(I.block(d, 16, 100 + r)).to(dev, dt))
            Ys.append(torch.empty_like(Xs[-1]))
        bound = [field_free_bound(m) for m in ms]
        pf.cheb_filter_batched(ms, [-b for b in bound], bound, [0.0] * n, [args.K] * n, Xs, Ys, 16, kind)
        torch.cuda.synchronize()
        print(f"filter-only ok: batched {args.workload} {args.precision} K={args.K}")
        return
    builder, L, W, n_ev, n_b, cfg = WORKLOADS[args.workload]
    m = builder(L, W, cfg, 0)
    dim = pf.basis_build(L, L // 2)
    st = torch.empty(dim, dtype=torch.int32, device=dev)
    pf.basis_build(L, L // 2, st)
    X = torch.from_numpy(I.block(dim, n_b, 7)).to(dev, dt)
    Y = torch.empty_like(X)
    b = field_free_bound(m)
    reps = max(1, args.reps)
    stream = torch.cuda.Stream(device=dev)  # a capturable stream (the Clenshaw loop may run as a CUDA graph)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0 = pf.get_counters()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(reps):
        pf.cheb_filter(m, st, dim, -b, b, 0.0, args.K, X, Y, n_b, kind, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    c1 = pf.get_counters()
    k = {pf.F64: 0, pf.F32: 1, pf.DF64: 2}[kind]
    n = c1["kind_launches"][k] - c0["kind_launches"][k]
    g = c1["kind_gpu_s"][k] - c0["kind_gpu_s"][k]
    a = c1["kind_alg_bytes"][k] - c0["kind_alg_bytes"][k]
    print(json.dumps({"filter_only": args.workload, "precision": args.precision, "K": args.K, "n_b": n_b,
                      "dim": dim, "reps": reps, "call_ms": round(ev0.elapsed_time(ev1) / reps, 3),
                      "step_launches": int(n), "avg_step_us": round(1e6 * g / max(n, 1), 2),
                      "alg_gbs": round(a / max(g, 1e-12) / 1e9, 1),
                      "frac_of_peak": round(a / max(g, 1e-12) / 1e9 / peaks()[0], 4)}), flush=True)


def field_free_bound(m):
    """A bound on ||H|| for Eq. (1): each bond term is at most |J_l| (1/2 + |Delta|/4), each field term |h_i|/2."""
    nb1 = m.L if m.periodic else m.L - 1
    nb2 = m.L if m.periodic else m.L - 2
    return 1.01 * ((nb1 * abs(m.J1) + nb2 * abs(m.J2)) * (0.5 + abs(m.Delta) / 4) + 0.5 * float(np.abs(m.h).sum()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="L22_xxz_W3", choices=sorted(WORKLOADS) + sorted(BATCHED))
    ap.add_argument("--precision", default=None, choices=sorted(PREC),
                    help="filter arithmetic (default: f32 stage + refinement)")
    ap.add_argument("--dos", default="mlp", choices=sorted(DOS),
                    help="density-of-states rule for K (mlp: the learned predictor, trained before timing)")
    ap.add_argument("--batch-mode", default="batched", choices=["batched", "sequential"],
                    help="batched workloads: one polfed_eigs_batched call, or polfed_eigs per realization")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--filter-only", action="store_true", help="one filter call (kernel profiling)")
    ap.add_argument("--K", type=int, default=6, help="--filter-only: filter order")
    ap.add_argument("--reps", type=int, default=1, help="--filter-only: filter calls")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "f32"
    if args.warmup < 3 and not args.filter_only:
        print("warning: fewer than 3 warm-up steps; the number is not valid", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2005_09534_gb300 as pf

    if args.filter_only:
        run_filter_only(args, pf, torch, dev)
    elif args.workload in BATCHED:
        run_batched(args, pf, torch, dev, world, rank, local, dist)
    else:
        run_single(args, pf, torch, dev, world, rank, local, dist)


def timed_realization(k, world, rank):
    """Realization index of run k on this rank (ranks never share one)."""
    return k * world + rank


def warmup_realization(w, world, rank):
    """Realization index of warm-up run w on this rank (disjoint from timed ones)."""
    return 10_000 + w * world + rank


def reduce_ranks(torch, dev, dist, t_dev, wall_s, pairs, pairs_wall=None):
    """Max of the times and sum of the (credited) eigenpairs over ranks."""
    if pairs_wall is None:
        pairs_wall = pairs
    if not dist:
        return t_dev, wall_s, pairs, pairs_wall
    tt = torch.tensor([t_dev, wall_s], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pp = torch.tensor([pairs, pairs_wall], device=dev, dtype=torch.float64)
    dist.all_reduce(pp)
    return float(tt[0]), float(tt[1]), float(pp[0]), float(pp[1])


def train_predictor(pf, ctx, builder, L, W, cfg_id, n_real=48, steps=4000):
    """Train the spectral predictor on labels the library produces (Lanczos
    bounds, KPM counts) for n_real realizations at W' in [W/2, 3W/2] (field
    config 90, disjoint from the timed realizations).  Untimed setup."""
    from paper_2005_09534_gb300 import predictor
    t0 = time.perf_counter()
    models, Ws = [], []
    for k in range(n_real):
        w = W * (0.5 + ((0.6180339887498949 * (k + 1)) % 1.0))
        m = builder(L, w, 90, k)
        models.append(m)
        Ws.append(w)
    labels = predictor.labels_for(ctx, models)
    t1 = time.perf_counter()
    X, Y = predictor.dataset(models, Ws, labels)
    net = pf.MLP(L + 1, 128, 3, seed=7)
    loss, secs = predictor.fit(net, X, Y, steps=steps, lr=2e-3, batch=256)
    return net, {"train_realizations": n_real, "samples": int(X.shape[0]), "label_s": round(t1 - t0, 1),
                 "train_s": round(secs, 1), "train_steps": steps, "train_loss": round(float(loss), 4)}


def batched_models(spec, base_realization):
    n, Ls, Wc, Nc, cfg = spec
    ms, nev = [], []
    for r in range(n):
        L = Ls[r % len(Ls)]
        m = I.xxz(L, Wc[r % len(Wc)], cfg, base_realization + r)
        ms.append(m)
        nev.append(Nc[r % len(Nc)])
    return ms, nev


def run_batched(args, pf, torch, dev, world, rank, local, dist):
    """One step = one polfed_eigs_batched call over the 64-realization batch
    (autotuned block widths, one cooperative filter launch per round)."""
    spec = BATCHED[args.workload]
    opts = pf.opts_default()
    opts.precision = PREC[args.precision] if args.precision != "f64" else pf.DF64

    def solve(ms, nev):
        if args.batch_mode == "batched":
            return pf.eigs_batched(ms, 0.5, nev, n_b=0, opts=opts, device=local, allow_fail=True)
        # the same realizations one after another through polfed_eigs (comparison mode)
        evs, res, sts, status = [], [], [], []
        t0 = time.perf_counter()
        with pf.Ctx(local) as ctx:
            for m, n in zip(ms, nev):
                nb = 16 if n <= 100 else 32
                ev, r, st, rc = pf.eigs(ctx, m, 0.5, n, 0, nb, opts, allow_noconv=True)
                evs.append(ev)
                res.append(r)
                sts.append(st)
                status.append(rc)
        info = {"n_width16": sum(1 for n in nev if n <= 100), "n_width32": sum(1 for n in nev if n > 100),
                "n_width64": 0, "ctas_per_sm": 0, "rounds": sum(s["n_step_launches"] for s in sts), "t_tune": 0.0,
                "filter_gpu_s": sum(s["step_gpu_s"] for s in sts),
                "filter_alg_bytes": sum(s["step_alg_bytes"] for s in sts),
                "n_launches": sum(s["n_launches"] for s in sts), "t_total": time.perf_counter() - t0}
        return evs, res, sts, np.array(status), info, 0

    for w in range(args.warmup):
        ms, nev = batched_models(spec, 1000 * warmup_realization(w, world, rank))
        solve(ms, nev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    wall_s, dev_s, pairs = 0.0, 0.0, 0
    infos, statuses, max_rr, restarts, fallbacks = [], [], 0.0, 0, 0
    for k in range(args.steps):
        ms, nev = batched_models(spec, 1000 * timed_realization(k, world, rank))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        evs, res, sts, status, info, rc = solve(ms, nev)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        wall_s += dt
        dev_s += dt  # host-driven multi-stream run: the device is busy for the whole call
        for i, st in enumerate(sts):
            hn = max(abs(st["E_min"]), abs(st["E_max"]))
            if status[i] == 0:
                pairs += int(np.sum(res[i] <= 1e-8 * hn))
            max_rr = max(max_rr, float(np.max(res[i]) / hn) if len(res[i]) else 0.0)
            restarts += st["n_restarts"]
            fallbacks += st["fallback_df64"]
        statuses += [int(x) for x in status]
        infos.append(info)
        for i, st in enumerate(sts):
            hn = max(abs(st["E_min"]), abs(st["E_max"]))
            print(f"[batched] r{i} L={ms[i].L} W={ms[i].W} N_ev={nev[i]} status={int(status[i])} n_b={st['n_b']} "
                  f"K={st['K']} m={st['m']} refine={st['n_refine']} restarts={st['n_restarts']} "
                  f"fallback={st['fallback_df64']} maxres/|H|={st['max_resid'] / hn:.2e} t={st['t_total']:.2f}s",
                  file=sys.stderr)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop() if rank == 0 else None
    t_dev, wall_s, pairs_all, _ = reduce_ranks(torch, dev, dist, dev_s, wall_s, pairs)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    fg = sum(i["filter_gpu_s"] for i in infos)
    fa = sum(i["filter_alg_bytes"] for i in infos)
    achieved = fa / fg / 1e9 if fg > 0 else 0.0
    n, Ls, Wc, Nc, cfg = spec
    line = {"metric": METRIC, "value": round(pairs_all / t_dev, 4), "unit": "eigenpairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_dev / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": args.workload, "mode": args.batch_mode, "realizations": n, "L": list(Ls),
                       "W": list(Wc),
                       "N_ev": list(Nc), "eps": 0.5, "hamiltonian": "xxz",
                       "n_width16_32_64": [infos[-1]["n_width16"], infos[-1]["n_width32"], infos[-1]["n_width64"]],
                       "ctas_per_sm": infos[-1]["ctas_per_sm"], "rounds": [i["rounds"] for i in infos],
                       "tune_s": [round(i["t_tune"], 2) for i in infos], "restarts": restarts,
                       "fallback_df64": fallbacks, "status_nonzero": sum(1 for x in statuses if x != 0),
                       "max_resid_over_normH": max_rr, "parallelism": f"replicas x{world}",
                       "l2": "instances of 12870-48620 rows: filter working sets partly L2-resident, no flush"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": f"of {peak_kind}",
                         "kernel": "k_filter_batched (all realizations' Clenshaw steps, one cooperative launch)",
                         "alg_bytes_per_launch": fa / max(1, sum(i["rounds"] for i in infos)),
                         "avg_launch_us": round(1e6 * fg / max(1, sum(i["rounds"] for i in infos)), 1)},
            "e2e": {"value": round(pairs_all / wall_s, 4), "unit": "eigenpairs/s",
                    "h2d_bytes_per_step": sum(m.L * 8 for m in batched_models(spec, 0)[0]),
                    "d2h_bytes_per_step": 16 * sum(batched_models(spec, 0)[1])},
            "gpu_launches": int(sum(i["n_launches"] for i in infos)),
            "clocks": ck}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_batched_sample(ms, nev, sts)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
