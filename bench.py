#!/usr/bin/env python
"""Benchmark of the condensed-IPM hot path on GB300.

Metric: condense + Cholesky milliseconds per IPM iteration (FP64) on the seeded
10,000-bus lattice workload (1,000 generators: nu = 1,999 controls, nx = 18,999
states), the largest single-instance configuration, at the oracle's own
linearize-then-reduce iterate 3 (stored in tests/golden/grid10k_iterate.npz).
One step is one pass of the per-iteration hot path: model derivatives (A1-A3),
G_x refactorisation, multi-right-hand-side triangular solves over all nu
columns, K assembly, H = K Z and the condensed matrix (A4-A7), the condensed
right-hand side (A8), one Cholesky attempt (A9) and the step recovery (A10).
``value`` is A4-A9 (the metric); ``ms_per_step`` the whole step.

Z and H (339 MB each) exceed L2 (129 MB); a 256 MB buffer is still written on
the stream between timed steps, so the factors and K start cold too.  Device
time comes from CUDA events on the library's stream.  ``e2e`` times the same
step through opf_newton_step with pinned HOST buffers (copies inside).
``--impl reference`` times the CPU FP64 oracle on the host cores for the same
metric and workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402

METRIC = "condense+Cholesky ms/IPM iter"
KERNEL_NAMES = {32: "column-parallel", 64: "level-blocked", 96: "dataflow", 1: "staged x1", 2: "staged x2",
                4: "staged x4", 128: "level-blocked on clusters"}
UNIT = "ms/iter"
WORKLOAD = ("grid10k: 10,000-bus lattice, 1,000 generators, nu=1,999, nx=18,999, FP64, "
            "LinRed oracle iterate 3")
ITERATE = os.path.join(ROOT, "tests", "golden", "grid10k_iterate.npz")


def stored_iterate(path=ITERATE):
    """The oracle's LinRed iterate 3 of the 10,000-bus workload: x, u, lambda,
    y, Sigma, the full-space right-hand side r and the delta_w its inertia
    correction took."""
    z = np.load(path)
    nu = (len(z["w"]) - len(z["lam"]))
    sw = z["sig_w"]
    return dict(x=z["w"][nu:], u=z["w"][:nu], lam=z["lam"], y=z["y"], sig_u=sw[:nu], sig_x=sw[nu:],
                sig_s=z["sig_s"], r=z["r"]), float(z["delta"])


def synthetic_iterate(net, nx, nu, m, seed=2203):
    """Flat-start-like primal point with moderate multipliers and barrier terms."""
    rng = np.random.default_rng(seed)
    n_ns = net.nb - 1
    x = np.concatenate([0.02 * rng.standard_normal(n_ns), 1.0 + 0.01 * rng.standard_normal(net.nb - net.ng)])
    u = np.concatenate([np.clip(1.05, net.Vmin[net.gbus], net.Vmax[net.gbus]),
                        0.5 * (net.Pmin[1:] + net.Pmax[1:])])
    lam = 20.0 + rng.standard_normal(nx)
    y = 0.1 * rng.random(m)
    sig_u = rng.uniform(1.0, 10.0, nu)
    sig_x = np.where(np.arange(nx) < n_ns, 0.0, rng.uniform(1.0, 10.0, nx))
    sig_s = rng.uniform(1.0, 10.0, m)
    r = rng.standard_normal(nu + nx + 2 * m + nx)
    return dict(x=x, u=u, lam=lam, y=y, sig_u=sig_u, sig_x=sig_x, sig_s=sig_s, r=r)


def shard(n_units, rank, world):
    """The units (instances) one rank of `world` processes: every world-th one,
    so that each size class is spread over the ranks."""
    return list(range(rank, n_units, world))


def aggregate(t_local, units_local, dist=None, device=None):
    """(max of the ranks' times, sum of the ranks' units); plain values alone."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_local), int(units_local)
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    u = torch.tensor([int(units_local)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def measured_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/traffic.json, key "kernel@workload"), or None when the
    summary is missing or was taken from different kernel sources."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = rec.get(f"{kernel}@{workload}")
    if not ent:
        return None
    h = hashlib.sha256()
    for f in ent.get("sources", []):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != ent.get("sha256"):
        return None
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for ln in open(self.path):
            p = [c.strip() for c in ln.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(p[1]) for p in rows if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in rows if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in rows for i in range(4) if p[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_condense(net, it, delta, budget_s=15.0, max_reps=200):
    """Oracle condense + Cholesky per iteration at the same iterate (host
    cores): Kred = Z^T K Z by its definition (SciPy splu for S_x, BLAS for the
    dense products) and numpy's Cholesky of Kred + delta I.  Returns the median
    milliseconds and the number of evaluations."""
    from oracle import kkt, model
    lay = model.Layout(net)
    w = np.concatenate([it["u"], it["x"]])
    sw = np.concatenate([it["sig_u"], it["sig_x"]])
    _, G, A = model.jacobians(lay, w)
    W = model.lagrangian_hessian(lay, w, it["lam"], it["y"])
    reps, t0 = 0, time.perf_counter()
    times = []
    while time.perf_counter() - t0 < budget_s or reps < 1:
        t2 = time.perf_counter()
        K = kkt.kred_definition(G, A, W, sw, it["sig_s"], lay.nu)
        np.linalg.cholesky(K + delta * np.eye(lay.nu))
        times.append((time.perf_counter() - t2) * 1e3)
        reps += 1
        if reps >= max_reps:
            break
    return float(np.median(times)), reps


def run_batch(binding, nthreads, rank=0, world=1, dist=None, device=None):
    """OPF solves/s of the 96 uneven instances (32 each at 500 / 1,500 / 3,000
    buses, loads scaled per bus): one at a time versus opf_batch_solve in
    lockstep (one batched condensation per iteration for every instance still
    iterating) and as concurrent independent loops, on the same handles after
    the batch autotuner picked their solve kernels.  Every batched objective is
    compared with its single-instance objective.  Also one condense + Cholesky
    of all instances at once (opf_batch_condense_factor) against the same work
    one instance at a time.  With several ranks each solves its shard of the
    instances (no collective on the data path); the rates are the instances of
    all ranks over the slowest rank's time."""
    import torch
    t00 = time.perf_counter()
    every = gridgen.batch96()
    nets = [every[i] for i in shard(len(every), rank, world)]
    hs = [binding.Handle(n, route=binding.OPF_ROUTE_AUTO) for n in nets]
    t01 = time.perf_counter()
    b = binding.Batch(hs, nthreads=nthreads)
    b.autotune()
    t02 = time.perf_counter()
    hs[0].solve()                    # warm-up: first-call costs out of the timing
    t0 = time.perf_counter()
    single = [h.solve() for h in hs]
    t_single = time.perf_counter() - t0
    b.set_mode("lockstep")
    batched, wall_ms = b.solve()
    t_batch = wall_ms * 1e-3
    b.set_mode("concurrent")
    conc, wall_c = b.solve()
    t_conc = wall_c * 1e-3
    rel = max(abs(a["obj"] - c["obj"]) / abs(a["obj"]) for a, c in zip(single, batched))
    rel_c = max(abs(a["obj"] - c["obj"]) / abs(a["obj"]) for a, c in zip(single, conc))
    ok = all(a["status"] == 0 and c["status"] == 0 and d["status"] == 0 for a, c, d in zip(single, batched, conc))
    # one condensation + Cholesky of every instance: batched vs one at a time
    pts = [synthetic_iterate(n, h.nx, h.nu, h.m, seed=7 + k) for k, (n, h) in enumerate(zip(nets, hs))]
    Ds = [{k: torch.as_tensor(v, dtype=torch.float64, device=device) for k, v in p.items()} for p in pts]
    for h, D in zip(hs, Ds):
        h.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
    deltas = []
    for h, D in zip(hs, Ds):
        h.condense(D["sig_u"], D["sig_x"], D["sig_s"])
        dl = 0.0
        while h.kkt_factor(dl) >= 0:
            dl = max(1e-4, 8 * dl)
        deltas.append(dl)
    sig = [[D["sig_u"] for D in Ds], [D["sig_x"] for D in Ds], [D["sig_s"] for D in Ds]]
    b.condense_factor(*sig, delta_w=deltas)          # builds the work lists
    reps = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        st, _ = b.condense_factor(*sig, delta_w=deltas)
    t_bcf = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        for h, D, dl in zip(hs, Ds, deltas):
            h.condense(D["sig_u"], D["sig_x"], D["sig_s"])
            h.kkt_factor(dl)
    t_scf = (time.perf_counter() - t0) / reps
    t_single, n_all = aggregate(t_single, len(nets), dist, device)
    t_batch, _ = aggregate(t_batch, len(nets), dist, device)
    t_conc, _ = aggregate(t_conc, len(nets), dist, device)
    out = {"instances": n_all, "sizes": "32 x 500 + 32 x 1,500 + 32 x 3,000 buses",
           "solves_per_s_single": n_all / t_single, "solves_per_s_batched": n_all / t_batch,
           "solves_per_s_concurrent": n_all / t_conc,
           "speedup": t_single / t_batch, "speedup_concurrent": t_single / t_conc,
           "wall_s_single": t_single, "wall_s_batched": t_batch, "wall_s_concurrent": t_conc,
           "batched_mode": "lockstep: one opf_batch_condense_factor per iteration for every instance still "
                           "iterating (one host thread per instance)",
           "lockstep_condensations": b.lockstep_calls(),
           "host_threads_concurrent": b.nthreads, "all_converged": ok,
           "max_rel_obj_diff_batched_vs_single": rel, "max_rel_obj_diff_concurrent_vs_single": rel_c,
           "iters_total": int(sum(c["iters"] for c in batched)),
           "iters_max": int(max(c["iters"] for c in batched)),
           "condense_factor_all_instances_ms": {"batched": t_bcf * 1e3, "one_at_a_time": t_scf * 1e3,
                                                "speedup": t_scf / t_bcf,
                                                "all_pd": all(v == 0 for v in st)}}
    # the condensation route each instance's autotuner picked, per size class
    routes = {}
    for n, h in zip(nets, hs):
        r, ms = h.route_choice()
        cls = routes.setdefault(str(n.nb), {"adjoint": 0, "explicit": 0, "ms_adjoint": [], "ms_explicit": []})
        cls["adjoint" if r == 0 else "explicit"] += 1
        cls["ms_adjoint"].append(ms["adjoint"])
        cls["ms_explicit"].append(ms["explicit"])
    for cls in routes.values():
        cls["ms_adjoint"] = float(np.median(cls["ms_adjoint"]))
        cls["ms_explicit"] = float(np.median(cls["ms_explicit"]))
    out["route_autotune"] = routes
    out["batch_tuning"] = b.stats()
    t03 = time.perf_counter()
    b.close()
    del hs
    out["setup_s"] = {"create": t01 - t00, "batch_and_autotune": t02 - t01, "teardown": time.perf_counter() - t03}
    return out


def run_reference(args):
    """The oracle as the reference arm: same metric, workload and unit; one
    oracle evaluation of condense + Cholesky at the stored iterate per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    net = gridgen.grid10k()
    it, delta = stored_iterate()
    for _ in range(args.warmup):
        cpu_oracle_condense(net, it, delta, budget_s=0.0)
    per = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ms, _ = cpu_oracle_condense(net, it, delta, budget_s=0.0)
        per.append(ms)
    wall = time.perf_counter() - t0
    value = float(np.mean(per))
    threads = os.environ.get("OMP_NUM_THREADS")
    cores = int(threads) if threads and threads.isdigit() else os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, args.steps),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{args.steps} oracle condense+Cholesky evaluations of the stored grid10k "
                                      "iterate (SciPy splu for S_x, serial; BLAS dense products and Cholesky)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def fp64_peaks(binding, torch, dev):
    """Measured FP64 throughput (GFLOP/s) of this GPU: the library's DFMA and
    f64 mma.sync probes, and torch's f64 matmul and Cholesky for context."""
    out = {}
    for k, name in enumerate(("dfma", "dmma_m8n8k4", "dmma_m16n8k4", "dmma_m16n8k16")):
        out[name] = binding.fp64_peak(k)
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    spd = a @ a.T + n * torch.eye(n, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn, fl in (("torch_matmul_4096", lambda: a @ b, 2.0 * n ** 3),
                         ("torch_cholesky_4096", lambda: torch.linalg.cholesky(spd), n ** 3 / 3.0)):
        fn()
        best = 1e30
        for _ in range(3):
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = fl / (best * 1e-3) / 1e9
    del a, b, spd
    return out


def path_flops(h):
    """Algorithmic FP64 flop of one condense + Cholesky (A4-A9, adjoint route,
    N = nu columns): four triangular solves over nu columns with the factors'
    strict parts (2 S nu each) and their diagonal scaling (nx nu per pair), the
    numeric LU (2 x the symbolic multiply-add count), H = K Z (2 nnz(K) nu),
    G_u^T Psi (2 nnz(G_u) nu) and the Cholesky (nu^3 / 3)."""
    st = h.stats()
    S = (st["nnz_lu"] - h.nx) // 2
    _, _, _, ci = h.get_csr_pattern(0)        # G = [G_u G_x], columns [u; x]
    nnz_gu = int((ci < h.nu).sum())
    trsm = 4 * 2 * S * h.nu + 2 * h.nx * h.nu
    # the forward sweep over P G_u on the level-blocked kernels solves, in each
    # full 32-column block, only the rows of its reach list: that sweep's share
    # of the count above, scaled by the listed fraction of those blocks' work
    nblk, work = h.forward_reach()
    kern = h.trsm_choice()[0]
    if nblk > 0 and kern in (64, 128) and work["all"] > 0:
        sweep = 2 * S * h.nu + h.nx * h.nu / 2
        trsm -= sweep * (32 * nblk / h.nu) * (1.0 - work["listed"] / work["all"])
    return {"trsm": trsm, "refactor": 2 * st["lu_flops"], "spmm": 2 * st["nnz_k"] * h.nu,
            "kred": 2 * nnz_gu * h.nu, "chol": h.nu ** 3 / 3.0, "S": S}


def time_condense(h, D, delta, reps, stream, torch):
    """Mean CUDA-event ms of condense + Cholesky (after one untimed pass)."""
    ts = []
    for k in range(reps + 1):
        h.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.condense(D["sig_u"], D["sig_x"], D["sig_s"])
        h.kkt_factor(delta)
        b.record(stream)
        b.synchronize()
        if k:
            ts.append(a.elapsed_time(b))
    return float(np.mean(ts))


def run_decay(binding, net, it, D, torch):
    """The decay of the reduced Hessian with the bus distance between controls
    (the structure Sec. 5 proposes to exploit), measured on the library's own
    Kred and reduced gradient at the grid10k iterate: normalised entries
    |K_ij| / sqrt(K_ii K_jj) by hop distance for the voltage and the dispatch
    controls, with and without the rank-one coupling through the slack
    generator (coefficient 2 c2_0 + Sigma_s,0 on v = Z^T grad P_slack), and the
    error of a probing approximation (distance-2d colouring, entries kept within
    distance d)."""
    import scipy.sparse as sps
    from scipy.sparse.csgraph import shortest_path
    h = binding.Handle(net)
    nu, nw = h.nu, h.nw
    h.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
    K = torch.zeros(nu * nu, dtype=torch.float64, device=D["x"].device)
    h.condense(D["sig_u"], D["sig_x"], D["sig_s"], K)
    K = K.cpu().numpy().reshape(nu, nu)
    K = 0.5 * (K + K.T)
    nr, nc, rp, ci = h.get_csr_pattern(binding.OPF_MAT_A)
    av = torch.zeros(len(ci), dtype=torch.float64, device=D["x"].device)
    h.get_csr_values(binding.OPF_MAT_A, av)
    av = av.cpu().numpy()
    a0 = np.zeros(nw)
    a0[ci[rp[0]:rp[1]]] = av[rp[0]:rp[1]]
    v = torch.zeros(nu, dtype=torch.float64, device=D["x"].device)
    h.reduced_gradient(torch.as_tensor(a0, device=D["x"].device), v)
    v = v.cpu().numpy()
    del h
    ng = net.ng
    busu = np.concatenate([net.gbus, net.gbus[1:]])
    graph = sps.coo_matrix((np.ones(net.nl), (net.lf, net.lt)), shape=(net.nb, net.nb))
    srcs = np.unique(busu)
    hop = shortest_path(graph, directed=False, unweighted=True, indices=srcs)
    row = {b: k for k, b in enumerate(srcs)}
    Dh = hop[np.array([row[b] for b in busu])][:, busu]
    coef = 2.0 * float(net.c2[0]) + float(it["sig_s"][0])

    def profile(M, idx):
        dg = np.sqrt(np.abs(np.diag(M)))
        Nm = np.abs(M) / np.outer(dg, dg)
        Nb, Db = Nm[np.ix_(idx, idx)], Dh[np.ix_(idx, idx)]
        return {int(k): [float(np.median(Nb[Db == k])), float(np.percentile(Nb[Db == k], 99))]
                for k in range(0, 31, 3) if (Db == k).any()}
    vm, pg = np.arange(ng), np.arange(ng, nu)
    K1 = K - coef * np.outer(v, v)
    probe = {}
    for d in (4, 8, 12):
        order = np.argsort(-np.sum(Dh <= 2 * d, axis=1), kind="stable")
        color = -np.ones(nu, int)
        for j in order:
            used = set(color[(Dh[j] <= 2 * d) & (color >= 0)].tolist())
            c = 0
            while c in used:
                c += 1
            color[j] = c
        nc_ = int(color.max()) + 1
        V = np.zeros((nu, nc_))
        V[np.arange(nu), color] = 1.0
        Kd = np.where(Dh <= d, (K @ V)[:, color], 0.0)
        Kd = 0.5 * (Kd + Kd.T)
        probe[d] = {"colors": nc_, "rel_err": float(np.linalg.norm(Kd - K) / np.linalg.norm(K))}
    return {"workload": "grid10k iterate: Kred and the slack row's reduced gradient from the library",
            "normalised_by_hops_median_p99": {"Vm-Vm": profile(K, vm), "Pg-Pg": profile(K, pg),
                                              "Vm-Vm_without_slack_rank1": profile(K1, vm),
                                              "Pg-Pg_without_slack_rank1": profile(K1, pg)},
            "probing": probe}


def run_fullspace(binding, net, it, delta, D, stream, flush, torch, split, no_solve, reps=20):
    """The hybrid full-space IPM's linear algebra (Sec. 4.3, Table 2's comparison
    method) on the same grid10k iterate: assembly + block LDL^T + inertia, then
    the step, CUDA events on the handle's stream with an L2 flush before each
    repetition; and whole solves of both IPMs."""
    hf = binding.Handle(net)
    hf.set_stream(stream)
    step = torch.zeros(hf.n_kkt, dtype=torch.float64, device=D["x"].device)
    for _ in range(3):
        hf.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
        rc, inert = hf.fullspace_factor(D["sig_u"], D["sig_x"], D["sig_s"], delta_w=delta)
        hf.fullspace_solve(D["r"], step, 1, 0)
    assert rc == binding.OPF_OK, inert
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    hf.profile(True)
    for k in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
        hf.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
        ev[k][0].record(stream)
        hf.fullspace_factor(D["sig_u"], D["sig_x"], D["sig_s"], delta_w=delta)
        ev[k][1].record(stream)
        hf.fullspace_solve(D["r"], step, 1, 0)
        ev[k][2].record(stream)
        steps, res = hf.fullspace_solve(D["r"], step, 1, 3)
        ev[k][3].record(stream)
    torch.cuda.synchronize()
    ph = hf.phase_times()
    hf.profile(False)
    st = hf.fullspace_stats()
    t_fac = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    t_sol = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    t_ref = float(np.mean([e[2].elapsed_time(e[3]) for e in ev]))
    linred = split["condense_cholesky"] + split["condensed_rhs"] + split["step_recovery"]
    out = {"workload": "grid10k stored iterate: augmented system with the slack step eliminated, "
                       f"{hf.nw + hf.nx + hf.m} unknowns, {st['nblocks']} diagonal blocks",
           "factor_ms": t_fac, "solve_ms": t_sol, "solve_refined_ms": t_ref, "refine_steps": steps,
           "refined_rel_residual": res, "per_iteration_ms": t_fac + t_sol,
           "linred_per_iteration_ms": linred, "linred_over_fullspace": linred / (t_fac + t_sol),
           "phases_ms_per_rep": {p: v[0] / reps for p, v in ph.items() if v[0] > 0},
           "inertia": list(inert), "block_levels": st["levels"], "nnz_l": st["nnz_l"],
           "tuning": hf.fullspace_tuning(),
           "factor_gflops": 2.0 * st["flops"] / (ph["chol"][0] / reps * 1e-3) / 1e9,
           "note": "LinRed's per-iteration linear algebra = condense + Cholesky + condensed RHS + step recovery "
                   "(split_ms_per_step); the hybrid's = assembly + block LDL^T + inertia + one solve"}
    del hf
    if not no_solve:
        for name, mk in (("grid2000", gridgen.grid2000), ("grid10k", gridgen.grid10k)):
            row = {}
            for ls in ("condensed", "fullspace"):
                hs = binding.Handle(mk())
                hs.set_stream(stream)
                t0 = time.perf_counter()
                r = hs.solve("linred", linear_solver=ls)
                row[ls] = {"wall_s": time.perf_counter() - t0, "iters": r["iters"], "obj": r["obj"],
                           "status": r["status"], "ms_condense_or_factor": r["ms_condense"] + r["ms_factor"],
                           "ms_solve": r["ms_solve"]}
                del hs
            row["rel_obj_diff"] = abs(row["condensed"]["obj"] - row["fullspace"]["obj"]) / abs(row["condensed"]["obj"])
            out[f"solve_{name}"] = row
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the 2,000-bus measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 96-instance batched solves")
    ap.add_argument("--no-solve", action="store_true", help="skip the whole-solve timing")
    ap.add_argument("--no-vjp", action="store_true", help="skip the 10,000-bus dispatch-derivative timing")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FP64 peak probes (derived peak instead)")
    ap.add_argument("--no-fullspace", action="store_true", help="skip the hybrid full-space comparison")
    ap.add_argument("--no-decay", action="store_true", help="skip the reduced-Hessian decay study")
    ap.add_argument("--batch-threads", type=int, default=0, help="host threads of the batch (0 = auto)")
    ap.add_argument("--workload", default="grid10k", choices=["grid10k", "grid2000"],
                    help="network of the timed loop: grid10k (the bench line, at the stored oracle iterate) or "
                         "grid2000 (for profiling the 2,000-bus case, at a synthetic iterate)")
    ap.add_argument("--chol-form", type=int, default=0, choices=[0, 1, 2],
                    help="dense Cholesky of Kred: 0 autotune, 1 barrier form, 2 dataflow form")
    ap.add_argument("--rhs-block", type=int, default=0, choices=[0, 1, 2, 4, 32, 64, 96, 128],
                    help="multi-RHS solve kernel (opf_options.rhs_block; 0 autotune)")
    ap.add_argument("--rhs1-kernel", type=int, default=0, choices=[0, 1, 64, 65, 66],
                    help="one-RHS solve kernel (opf_options.rhs1_kernel; 0 autotune)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2203_11875_gb300 import binding, build
    build.build()
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    peaks = None if args.no_peaks else fp64_peaks(binding, torch, dev)
    sm_max = 2070.0
    try:
        sm_max = float(subprocess.run(["nvidia-smi", f"--id={local}", "--query-gpu=clocks.max.sm",
                                       "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                      timeout=30).stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    derived = props.multi_processor_count * 2 * 2 * sm_max / 1e3   # SMs x DFMA/clk x flop x GHz
    # the best FP64 rate the device delivers among the probes (DFMA and the f64
    # mma.sync shapes measure within a few per cent of each other)
    peak = max(peaks[k] for k in ("dfma", "dmma_m8n8k4", "dmma_m16n8k4", "dmma_m16n8k16")) if peaks else derived
    net = gridgen.grid10k() if args.workload == "grid10k" else gridgen.grid2000()
    h = binding.Handle(net, chol_form=args.chol_form, rhs_block=args.rhs_block, rhs1_kernel=args.rhs1_kernel)
    stream = torch.cuda.Stream(device=dev)
    h.set_stream(stream)
    if args.workload == "grid10k":
        it, delta = stored_iterate()
    else:
        it, delta = synthetic_iterate(net, h.nx, h.nu, h.m), 0.0
    D = {k: torch.as_tensor(v, dtype=torch.float64, device=dev) for k, v in it.items()}
    step = torch.zeros(h.n_kkt, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def hot_step(dl):
        h.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
        h.condense_rhs(D["sig_u"], D["sig_x"], D["sig_s"], D["r"])
        return h.kkt_factor(dl)

    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 3)):
        while hot_step(delta) >= 0:
            delta = max(1e-4, 8 * delta)
        h.kkt_solve_condensed(step)
    torch.cuda.synchronize()
    trsm_kernel, trsm_tune, trsm_kernel1 = h.trsm_choice()
    chol_form, chol_grid, chol_tune = h.chol_choice()
    cs_cluster, cs_tune = h.chol_solve_choice()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    h.profile(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = binding.launch_count()
    sampler.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
        h.eval_derivatives(D["x"], D["u"], D["lam"], D["y"])
        ev[k][1].record(stream)
        # A4-A9: condensation with the step's right-hand side as one extra column
        h.condense_rhs(D["sig_u"], D["sig_x"], D["sig_s"], D["r"])
        assert h.kkt_factor(delta) == -1
        ev[k][2].record(stream)
        h.kkt_solve_condensed(step)
        ev[k][3].record(stream)
    torch.cuda.synchronize()
    n_launch = binding.launch_count() - n_launch0
    clocks = sampler.stop()
    phases = h.phase_times()
    h.profile(False)
    cf = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    full = [ev[k][0].elapsed_time(ev[k][3]) for k in range(args.steps)]
    ph = {p: v[0] / args.steps for p, v in phases.items()}
    split = {"eval": float(np.mean([ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)])),
             "condense_cholesky": float(np.mean(cf)),
             "condensed_rhs": ph["rhs"],
             "step_recovery": float(np.mean([ev[k][2].elapsed_time(ev[k][3]) for k in range(args.steps)]))}
    t_cf = float(np.mean(cf)) + ph["rhs"]      # A4-A9: condensation, Cholesky and the condensed RHS
    t_full = float(np.mean(full))
    if dist:
        t = torch.tensor([t_cf, t_full], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_cf, t_full = t.tolist()
    # roofline of the dominant kernel: the multi-RHS triangular solves
    fl = path_flops(h)
    trsm_ms, trsm_n = phases["trsm"]
    per_launch_ms = trsm_ms / max(1, trsm_n)
    launches_per_step = trsm_n / args.steps          # 4 (one triangle each) or 2 (both triangles)
    flops_per_launch = fl["trsm"] / max(1.0, launches_per_step)
    achieved = flops_per_launch / (per_launch_ms * 1e-3) / 1e9 if trsm_n else None
    trsm_base = {32: "k_trsm_cols", 64: "k_trsm_blk", 96: "k_trsm_df", 128: "k_trsm_blkc"}.get(
        trsm_kernel, f"k_trsm_st<{trsm_kernel}>")
    trsm_name = trsm_base + {32: " (column-parallel)", 64: " (level-blocked)", 96: " (dataflow)",
                             128: " (level-blocked, clusters)"}.get(trsm_kernel, " (staged)")
    traffic = measured_traffic(trsm_base, args.workload)
    fl_path = sum(v for k, v in fl.items() if k != "S")
    cf_ms = float(np.mean(cf))
    # end to end through the public API with pinned host buffers: opf_newton_step
    keys = ("x", "u", "lam", "y", "sig_u", "sig_x", "sig_s", "r")
    host = {k: torch.as_tensor(it[k], dtype=torch.float64).pin_memory() for k in keys}
    step_h = torch.zeros(h.n_kkt, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in host.values())
    d2h = step_h.numel() * 8
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e2e = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
        assert h.newton_step(*[host[k_] for k_ in keys], step_h, delta_w=delta) == -1
        with torch.cuda.stream(stream):
            e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
    e2e_ms = float(np.mean(e2e))
    step_dev = step.cpu().numpy()
    e2e_rel = float(np.abs(step_h.numpy() - step_dev).max() / max(np.abs(step_dev).max(), 1e-300))
    out = {"metric": METRIC, "value": t_cf, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_full, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.workload == "grid10k" else
                      "grid2000: 2,000-bus lattice, 200 generators, nu=399, nx=3,799, FP64, synthetic iterate",
                      "inputs": "tests/golden/grid10k_iterate.npz (oracle LinRed iterate 3 of the seeded 10,000-bus "
                                "network)" if args.workload == "grid10k" else "bench.synthetic_iterate(grid2000)",
                      "l2": ("inputs larger than L2 (Z, H 339 MB each) and " if args.workload == "grid10k" else "")
                      + "a 256 MB flush written between timed steps",
                      "timed": "A4-A9: G_x refactor, multi-RHS solves (the step's right-hand side as one extra "
                               "column), K, H = K Z, Kred and the condensed right-hand side, one Cholesky attempt "
                               "(events) + reading the condensed right-hand side out (phase events)",
                      "route": "adjoint", "delta_w": delta,
                      "rhs_width": {"N": h.rhs_width()[0],
                                    "autotune_ms_at_nu_512_256_128": h.rhs_width()[1]},
                      "trsm_kernel": KERNEL_NAMES.get(trsm_kernel, str(trsm_kernel)),
                      "trsm_kernel_1rhs": KERNEL_NAMES.get(trsm_kernel1, str(trsm_kernel1)),
                      "autotune_ms": trsm_tune,
                      "cholesky": {"form": {1: "barrier", 2: "dataflow"}.get(chol_form, str(chol_form)),
                                   "ctas": chol_grid, "autotune_ms": chol_tune,
                                   "solve_cluster": cs_cluster,
                                   "solve_cluster_autotune_ms": {str(c): v for c, v in cs_tune.items()}}},
           "clocks": clocks, "gpu_launches": int(n_launch),
           "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "includes": "opf_newton_step from pinned host buffers: H2D of x, u, lambda, y, Sigma, r + "
                               "derivatives + condense + Cholesky + step solve and recovery + D2H of the step",
                   "max_rel_diff_vs_device_step": e2e_rel},
           "split_ms_per_step": split,
           "phases_ms_per_step": ph,
           "roofline": {"bound": "alu", "kernel": trsm_name,
                        "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                        "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                        "flops_per_launch": flops_per_launch, "ms_per_launch": per_launch_ms,
                        "launches_per_step": launches_per_step,
                        "peak_note": ("FP64 measured live in this run: the best of opf_fp64_peak's DFMA and f64 "
                                      "mma.sync probes (fp64_peaks_gflops); the measured-peak file has no FP64 entry"
                                      if peaks else
                                      "FP64 derived: SMs x 2 DFMA/clk x 2 flop x max SM clock"),
                        "peak_derived": derived},
           "path_roofline": {"flops": fl_path, "ms": cf_ms, "achieved": fl_path / (cf_ms * 1e-3) / 1e9,
                             "peak": peak, "frac": fl_path / (cf_ms * 1e-3) / 1e9 / peak,
                             "flops_by_phase": {k: v for k, v in fl.items() if k != "S"},
                             "note": "algorithmic FP64 flop of condense + Cholesky (adjoint route) over its "
                                     "CUDA-event time, against the measured FP64 peak"},
           "fp64_peaks_gflops": peaks,
           "symbolic": h.stats()}
    if world > 1:
        out["value"] = t_cf / world
    if not args.no_small:
        n2 = gridgen.grid2000()
        h2 = binding.Handle(n2, chol_form=args.chol_form)
        h2.set_stream(stream)
        i2 = synthetic_iterate(n2, h2.nx, h2.nu, h2.m)
        D2 = {k: torch.as_tensor(v, dtype=torch.float64, device=dev) for k, v in i2.items()}
        d2 = 0.0
        for _ in range(3):
            h2.eval_derivatives(D2["x"], D2["u"], D2["lam"], D2["y"])
            h2.condense(D2["sig_u"], D2["sig_x"], D2["sig_s"])
            while h2.kkt_factor(d2) >= 0:
                d2 = max(1e-4, 8 * d2)
        h2.profile(True)
        t2 = time_condense(h2, D2, d2, 20, stream, torch)
        ph2 = h2.phase_times()
        h2.profile(False)
        k2, tune2, _ = h2.trsm_choice()
        cf2, cg2, ct2 = h2.chol_choice()
        out["grid2000"] = {"workload": "grid2000: nu=399, nx=3,799, synthetic flat-start-like iterate",
                           "condense_cholesky_ms": t2, "trsm_kernel": KERNEL_NAMES.get(k2, str(k2)),
                           "cholesky": {"form": cf2, "ctas": cg2},
                           "phases_ms_per_step": {p: v[0] / 21 for p, v in ph2.items()}}
        del h2
    if not args.no_vjp:
        # the dispatch derivative of the converged 10,000-bus solve for 256 unit cotangents
        r10 = h.solve("linred")
        V = torch.as_tensor(gridgen.cotangents(net.ng), dtype=torch.float64, device=dev)
        gP = torch.empty((V.shape[0], net.nb), dtype=torch.float64, device=dev)
        gQ = torch.empty_like(gP)
        t0 = time.perf_counter()
        h.vjp_prepare()
        t_prep = time.perf_counter() - t0
        h.dispatch_vjp(V, gP, gQ)                    # warm-up (workspace growth)
        reps = []
        for _ in range(3):
            t0 = time.perf_counter()
            h.dispatch_vjp(V, gP, gQ)
            reps.append(time.perf_counter() - t0)
        info = h.vjp_info()
        out["vjp_grid10k"] = {"cotangents": int(V.shape[0]), "solve_s": r10["ms_total"] * 1e-3,
                              "solve_iters": r10["iters"], "solve_obj": r10["obj"], "prepare_ms": t_prep * 1e3,
                              "vjp_ms": float(np.median(reps)) * 1e3, "refine_steps": info["refine_steps"],
                              "rel_residual": info["rel_residual"], "polish_iters": info["polish_iters"]}
    if not args.no_decay:
        out["reduced_hessian_decay"] = run_decay(binding, net, it, D, torch)
    if not args.no_fullspace:
        out["hybrid_fullspace"] = run_fullspace(binding, net, it, delta, D, stream, flush, torch,
                                                out["split_ms_per_step"], args.no_solve)
    if not args.no_batch:
        out["batch96"] = run_batch(binding, args.batch_threads, rank, world, dist, dev)
    # one whole interior-point solve of the 2,000-bus network (LinRed), GPU path
    if not args.no_solve:
        n2 = gridgen.grid2000()
        hs = binding.Handle(n2)
        hs.set_stream(stream)
        t0 = time.perf_counter()
        rs = hs.solve("linred")
        out["solve"] = {"workload": "grid2000 LinRed from the flat start", "wall_s": time.perf_counter() - t0,
                        "iters": rs["iters"], "obj": rs["obj"], "status": rs["status"],
                        "graph_iters": rs["graph_iters"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ms, reps = cpu_oracle_condense(net, it, delta, budget_s=20.0)
        out["cpu_baseline"] = {"value": ms, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{reps} oracle condense+Cholesky evaluations of the stored grid10k "
                                         "iterate (SciPy splu for S_x runs on one thread; the BLAS products "
                                         "and the Cholesky on all host threads)"}
        # the same with BLAS pinned to one thread, in a child process
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        try:
            r1 = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                 "--steps", "2", "--warmup", "0"], env=env, capture_output=True, text=True,
                                timeout=600)
            one = json.loads(r1.stdout.strip().splitlines()[-1])
            out["cpu_baseline_1thread"] = {"value": one["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                           "sample": "2 oracle condense+Cholesky evaluations of the stored "
                                                     "grid10k iterate, BLAS on one thread"}
        except (subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
            out["cpu_baseline_1thread"] = {"unavailable": str(e)[:200]}
        if not args.no_solve:
            from oracle import ipm as oracle_ipm
            t0 = time.perf_counter()
            ro = oracle_ipm.linred(gridgen.grid2000())
            out["solve"]["cpu_oracle_wall_s"] = time.perf_counter() - t0
            out["solve"]["cpu_oracle_iters"] = ro.iters
            out["solve"]["rel_obj_diff_vs_oracle"] = abs(ro.obj - out["solve"]["obj"]) / abs(ro.obj)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
