"""Benchmark: BOUNCE vs BAOAB (1 fs) on a 4,096-molecule flexible-water
droplet (12,288 atoms, 12 A cutoff, cell list) on one GB300.

One "step" is one full integrator step (row-rebuild check, F_0 or the full
gradient, the two jump half-steps, B, A, O).  The headline value is BOUNCE
ns/day; BAOAB ns/day and pair evaluations per second ride along.

Protocol (our arm):
  * the droplet is pre-equilibrated on the GPU with BAOAB (friction 0.05/fs,
    1,500 steps) from the seeded lattice, so every timed window starts from
    a 300 K liquid droplet;
  * W warm-up steps, then the K timed steps run in windows of at most 5
    steps, each window restarting from the equilibrated state (the state is
    restored outside the timed region): BOUNCE with this split (bare-Coulomb
    jumps beyond 4-5 A) heats flexible water by ~15 % per 1 fs step (see the
    design notes), so each window measures steps of a droplet near 300 K;
  * L2 is flushed (a 256 MB write) before each timed window;
  * device time by CUDA events on the launch stream; nvidia-smi clocks are
    sampled during the timed windows;
  * e2e: the same windows through the public API with host buffers (state
    upload, run, state download), host wall clock;
  * roofline: the fused step kernel timed by CUDA events around each launch
    in a separate profiling pass of the same workload.
--impl reference times the FP64 oracle on the host cores on a bounded sample
(every 8th atom of the droplet per step; time scaled to all atoms).
Under torchrun (N > 1) every rank runs an independent replica (weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WINDOW = 5
N_SIDE = 16                  # 16^3 = 4096 molecules
R_CUT, R_ON, R_OFF, SKIN = 12.0, 4.0, 5.0, 1.0
DT = 1.0
# DRAM bytes (read + write) of one body launch of the BOUNCE step kernel with
# per-type-pair bounds on the 12,288-atom lattice droplet (82 proposals per
# atom-step; the timed windows run ~85): one ncu capture of the current kernel
K_STEP_TRAFFIC = 36794368 + 30464
# Algorithmic lane-operations per unit of work in the fused step kernel,
# counted from the kernel source:
OPS_PER_PROPOSAL = 150       # Philox4x32-10 (~100 int ops) + partner gather + FP32 pair term + decision
OPS_PER_SHORT_PAIR = 35      # FP32 pair term (displacement, r^2, rsqrt, chi, W'/r, accumulate)
OPS_PER_FULL_PAIR = 25       # FP32 pair term without the switching function


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_wait = time.perf_counter()
            while not self.samples and time.perf_counter() - t_wait < 5.0:   # sampler running before timing
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()
        t_wait = time.perf_counter()
        while not any(t >= self.t1 for t, _ in self.samples) and time.perf_counter() - t_wait < 1.0:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.perf_counter(), parts))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        """Samples taken while the timed region ran, plus the first one after it."""
        t0 = self.t0 if self.t0 is not None else -math.inf
        t1 = self.t1 if self.t1 is not None else math.inf
        inside = [p for t, p in self.samples if t0 <= t <= t1]
        after = [p for t, p in self.samples if t > t1][:1]
        samples = inside + after
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in samples if s[1].replace('.', '', 1).isdigit()]
        mx = [float(s[2]) for s in samples if s[2].replace('.', '', 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in samples for k in range(4) if s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(samples), "samples_inside_timed_region": len(inside)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def ns_per_day(steps, seconds):
    return steps * DT * 1e-6 * 86400.0 / seconds


def our_arm(args):
    import torch
    from paper_2002_07109_gb300 import bounce
    from paper_2002_07109_gb300.water import water_droplet

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    stream = torch.cuda.current_stream(device)
    sh = stream.cuda_stream
    s = water_droplet(N_SIDE, seed=rank)
    cfg = dict(r_on=R_ON, r_off=R_OFF, r_cut=R_CUT, skin=SKIN, dt=DT, device=local)
    # pre-equilibration
    eq = bounce.from_system(s, seed=1000 + rank, gamma=0.05, **cfg)
    eq.set_state(s.q, s.v)
    eq.run(1500, bounce.BAOAB, stream=sh)
    q0, v0 = eq.get_state()
    e_eq = eq.energies()
    eq.close()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)  # 256 MB > L2
    windows = [WINDOW] * (args.steps // WINDOW) + ([args.steps % WINDOW] if args.steps % WINDOW else [])
    res = {}
    # "bounce": per-type-pair bounds with the two-stage partner choice;
    # "bounce_rowmax": one bound per atom type, partner uniform over the row
    arms = (("bounce", bounce.BOUNCE, True), ("baoab", bounce.BAOAB, False),
            ("bounce_rowmax", bounce.BOUNCE, False))
    for name, integ, pb in arms:
        ctx = bounce.from_system(s, seed=7 + rank, pair_bounds=pb, **cfg)
        ctx.set_state(q0, v0, step=0)
        if args.warmup:
            ctx.run(args.warmup, integ, stream=sh)
        torch.cuda.synchronize()
        ctx.reset_counters(stream=sh)
        ms = 0.0
        launches = 0
        t_end = []
        with Clocks(local) as clk:
            _barrier(ws)
            torch.cuda.synchronize()
            clk.start()
            torch.cuda.nvtx.range_push(name + "_timed")
            for k, w in enumerate(windows):
                ctx.set_state(q0, v0, step=100000 * (k + 1))
                launches += ctx.run_launch_count(w, integ)
                flush.fill_(float(k))
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.run(w, integ, stream=sh)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
                t_end.append(ctx.energies(stream=sh)["temperature"])
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            clk.stop()
            _barrier(ws)
        e = ctx.energies(stream=sh)
        # e2e through the public API with host buffers
        t_e2e = 0.0
        for k, w in enumerate(windows):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_state(q0, v0, step=200000 * (k + 1))
            ctx.run(w, integ, stream=sh)
            qh, vh = ctx.get_state(stream=sh)
            t_e2e += time.perf_counter() - t0
        # kernel timing pass
        ctx.set_state(q0, v0, step=300000)
        ctx.reset_counters(stream=sh)
        kms, nl = ctx.profile_steps(min(args.steps, WINDOW), integ, stream=sh)
        ep = ctx.energies(stream=sh)
        res[name] = dict(ms=ms, clocks=clk.summary(), energies=e, t_end=t_end, e2e_s=t_e2e, kernel_ms=kms,
                         kernel_launches=nl, prof=ep,
                         launches=launches)
        ctx.close()
    steps = args.steps
    out = {}
    b, a = res["bounce"], res["baoab"]
    t_b = _max_over_ranks(b["ms"] / 1e3, ws, device)
    t_a = _max_over_ranks(a["ms"] / 1e3, ws, device)
    value = ws * ns_per_day(steps, t_b)
    baoab_value = ws * ns_per_day(steps, t_a)
    pe_b = _sum_over_ranks(b["energies"]["short_pairs"] + b["energies"]["proposals"], ws, device) / t_b
    pe_a = _sum_over_ranks(a["energies"]["full_pairs"], ws, device) / t_a
    # roofline of the fused BOUNCE step kernel: algorithmic lane-ops per launch / launch time
    prof = b["prof"]
    ops = OPS_PER_PROPOSAL * prof["proposals"] + OPS_PER_SHORT_PAIR * prof["short_pairs"]
    per_launch_s = b["kernel_ms"] / 1e3 / b["kernel_launches"]
    achieved = ops / b["kernel_launches"] / per_launch_s / 1e12
    clk = b["clocks"]
    sm_mhz = clk.get("sm_mhz") or 1995.0
    peak = 152 * 128 * sm_mhz * 1e6 / 1e12   # FP32/INT32 lane-ops per second at the sampled clock
    prof_a = a["prof"]
    ops_a = OPS_PER_FULL_PAIR * prof_a["full_pairs"]
    ach_a = ops_a / a["kernel_launches"] / (a["kernel_ms"] / 1e3 / a["kernel_launches"]) / 1e12
    n_atoms = 3 * N_SIDE ** 3
    h2d = 2 * n_atoms * 3 * 8
    e2e_val = ws * ns_per_day(steps, _max_over_ranks(b["e2e_s"], ws, device))
    line = {
        "metric": "ns/day & pair-evals/s, BOUNCE vs BAOAB 1fs on one GB300 at matched <E>, RDF",
        "value": round(value, 4),
        "unit": "ns/day",
        "n_gpus": ws,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_b * 1e3 / steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 pair math, f64 integration",
        "data": "synthetic: seeded lattice water droplet, BAOAB pre-equilibrated at 300 K",
        "config": {"workload": "BOUNCE (per-type-pair bounds), 4096-molecule flexible-water droplet (12288 atoms), r_c 12 A, "
                               "cell list, "
                               "switch 4-5 A, 1 fs, friction 1/ps",
                   "atoms": n_atoms, "windows_of_steps": WINDOW, "l2": "flushed before each timed window",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "baoab": {"value": round(baoab_value, 4), "unit": "ns/day", "ms_per_step": round(t_a * 1e3 / steps, 5),
                  "pair_evals_per_s": pe_a},
        "bounce_pair_evals_per_s": pe_b,
        "bounce_rowmax_bounds": {
            "value": round(ws * ns_per_day(steps, _max_over_ranks(res["bounce_rowmax"]["ms"] / 1e3, ws, device)), 4),
            "unit": "ns/day",
            "proposals_per_atom_step": res["bounce_rowmax"]["energies"]["proposals"] / (steps * n_atoms)},
        "speedup_vs_own_baoab": round(value / baoab_value, 4),
        "proposals_per_atom_step": b["energies"]["proposals"] / (steps * n_atoms),
        "accepts_per_atom_step": b["energies"]["accepts"] / (steps * n_atoms),
        "near_ties": b["energies"]["near_ties"],
        "temperature_end_of_windows_K": {"bounce": [round(x, 1) for x in b["t_end"]][:4],
                                         "baoab": [round(x, 1) for x in a["t_end"]][:4]},
        "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 3), "unit": "Tops/s",
                     "frac": round(achieved / peak, 4), "traffic": K_STEP_TRAFFIC,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one body launch of "
                                       "k_step<BOUNCE> on the same-size lattice droplet (per-type-pair bounds)",
                     "kernel": "k_step<BOUNCE> (fused F_0 + 2 jump half-steps + B A O A)",
                     "baoab_kernel_frac": round(ach_a / peak, 4)},
        "e2e": {"value": round(e2e_val, 4), "unit": "ns/day", "h2d_bytes_per_step": h2d * len(windows) // steps,
                "d2h_bytes_per_step": h2d * len(windows) // steps},
        "gpu_launches": b["launches"],
        "clocks": clk,
    }
    line["long_run"] = long_run(s, q0, v0, cfg, rank, stream, sh)
    line["pbc_box"] = pbc_box(rank, stream, sh)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(s)
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def long_run(s, q0, v0, cfg, rank, stream, sh, n_steps=1000, chunk=100):
    """Graph-captured runs of n_steps from the equilibrated state (after 64
    warm-up steps), for the matched-observables comparison: BAOAB; BOUNCE
    with the LJ part on the jumps and Coulomb in F_0 (per-type-pair bounds);
    BOUNCE with Coulomb and LJ on the jumps (the headline split), which heats
    and is reported with the step at which it stopped.  Each: ns/day over the
    chunks timed with CUDA events, and the means of the potential energy per
    molecule and of the temperature sampled after every chunk."""
    import torch
    from paper_2002_07109_gb300 import bounce
    n_mol = s.n_atoms // 3
    out = {}
    arms = (("baoab", bounce.BAOAB, dict(pair_bounds=False)),
            ("bounce_lj_jumps", bounce.BOUNCE, dict(pair_bounds=True, jump_coulomb=False)),
            ("bounce_coulomb_lj_jumps", bounce.BOUNCE, dict(pair_bounds=True)))
    for name, integ, extra in arms:
        ctx = bounce.from_system(s, seed=11 + rank, **cfg, **extra)
        ctx.set_state(q0, v0, step=0)
        ms, pe, T, done, err = 0.0, [], [], 0, None
        try:
            ctx.run(64, integ, stream=sh)
            torch.cuda.synchronize()
            ctx.reset_counters(stream=sh)
            for _ in range(n_steps // chunk):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.run(chunk, integ, stream=sh)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
                done += chunk
                e = ctx.energies(stream=sh)
                pe.append(e["potential"] / n_mol)
                T.append(e["temperature"])
        except Exception as ex:  # a blown-up state is reported, not timed
            err = str(ex).split("(")[0].strip()
        ctx.close()
        r = {"steps": done}
        if done:
            r.update({"ns_per_day": round(ns_per_day(done, ms / 1e3), 2), "pe_per_molecule": round(float(np.mean(pe)), 4),
                      "temperature_K": round(float(np.mean(T)), 1)})
        if err:
            r["stopped"] = err
        out[name] = r
    return out


def pbc_box(rank, stream, sh, n_steps=960, chunk=48):
    """The periodic box of 32,768 water molecules (98,304 atoms, edge 99.3 A):
    Ewald direct erfc (beta 0.35) and LJ within 9 A, SPME 96^3 of order 5,
    jumps beyond a 7.5-8.5 A switch (per-type-pair bounds), 1 fs, friction
    1/ps.  From a BAOAB-equilibrated state, graph-captured runs of n_steps
    after one warm-up chunk: BAOAB (SPME every step), BOUNCE-RESPA (SPME on
    the 2 fs outer step) and BOUNCE-RESPA1 (short-range pairs on 2 fs, SPME on
    6 fs).  ns/day over the chunks (CUDA events), and the means of the
    potential energy per molecule and of the temperature after every chunk."""
    import torch
    from paper_2002_07109_gb300 import bounce
    from paper_2002_07109_gb300.water import water_box
    s = water_box(32, seed=rank)
    n_mol = s.n_atoms // 3
    cfg = dict(r_on=7.5, r_off=8.5, r_cut=9.0, skin=1.0, dt=1.0, ewald_beta=0.35, pme_grid=(96, 96, 96),
               pme_order=5, max_neighbors=1024, max_short=640, device=torch.cuda.current_device())
    eq = bounce.from_system(s, seed=500 + rank, gamma=0.05, **cfg)
    eq.set_state(s.q, s.v)
    eq.run(600, bounce.BAOAB, stream=sh)
    q0, v0 = eq.get_state(stream=sh)
    eq.close()
    out = {"workload": "32,768-molecule periodic water box (98,304 atoms), erfc beta 0.35, r_c 9 A, SPME 96^3 order 5, "
                       "switch 7.5-8.5 A, 1 fs, friction 1/ps"}
    arms = (("baoab", bounce.BAOAB, dict(pair_bounds=False)),
            ("bounce_respa", bounce.BOUNCE_RESPA, dict(pair_bounds=True, respa_m=2)),
            ("bounce_respa1", bounce.BOUNCE_RESPA1, dict(pair_bounds=True, respa_m=2, respa_m2=3)))
    for name, integ, extra in arms:
        ctx = bounce.from_system(s, seed=21 + rank, **cfg, **extra)
        ctx.set_state(q0, v0, step=0)
        ms, pe, T, done, err = 0.0, [], [], 0, None
        try:
            ctx.run(chunk, integ, stream=sh)
            torch.cuda.synchronize()
            ctx.reset_counters(stream=sh)
            for _ in range(n_steps // chunk):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.run(chunk, integ, stream=sh)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
                done += chunk
                e = ctx.energies(stream=sh)
                pe.append(e["potential"] / n_mol)
                T.append(e["temperature"])
            props = ctx.energies(stream=sh)["proposals"]
        except Exception as ex:  # a blown-up state is reported, not timed
            err = str(ex).split("(")[0].strip()
        ctx.close()
        r = {"steps": done}
        if done:
            r.update({"ns_per_day": round(ns_per_day(done, ms / 1e3), 2), "pe_per_molecule": round(float(np.mean(pe)), 4),
                      "temperature_K": round(float(np.mean(T)), 1)})
            if integ != bounce.BAOAB and err is None:
                r["proposals_per_atom_step"] = round(props / (done * s.n_atoms), 4)
        if err:
            r["stopped"] = err
        out[name] = r
    return out


def _oracle_setup(s):
    from oracle.forcefield import Params
    from oracle.integrate import OracleMD, Topology
    topo = Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    p = Params(r_on=R_ON, r_off=R_OFF, r_cut=R_CUT, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps)
    return topo, p


def oracle_sample_step(md, sample):
    """One BJAOAJB step of the oracle restricted to the sampled atoms (the
    other atoms stay put): rows, F_0 and both jump half-steps for `sample`."""
    from oracle import philox
    from oracle.forcefield import ACCEL, pair_gradients, bonded_gradients
    from oracle.integrate import jump_half, o_step
    from oracle.neighbors import rows, to_pairs
    q, v, t, p = md.q, md.v, md.topo, md.p
    r = rows(q, t.mol, md.r_list, p.box, atoms=sample)
    ii, jj = to_pairs(r, sample)
    h = 0.5 * md.dt

    def g0():
        g = pair_gradients(q, t.charge, t.type, ii, jj, p, "short")[sample]
        return g + bonded_gradients(q, t.bonds, t.bond_k_r0, t.angles, t.angle_k_t0)[sample]

    full_rows = [np.zeros(0, np.int64)] * len(q)
    for a, i in enumerate(sample):
        full_rows[i] = r[a]
    vs = v.copy()
    vs[sample] -= (h * ACCEL / t.mass[sample])[:, None] * g0()
    vs, _ = jump_half(q, vs, full_rows, t, p, md.Lstar, md.beta, md.dt, md.seed, md.step_index, philox.STREAM_J1,
                      pair_bounds=md.pair_bounds)
    q[sample] += h * vs[sample]
    vs[sample] = o_step(vs[sample], t.mass[sample], md.T, md.gamma, md.dt, md.seed, md.step_index, atoms=sample)
    q[sample] += h * vs[sample]
    vs, _ = jump_half(q, vs, full_rows, t, p, md.Lstar, md.beta, md.dt, md.seed, md.step_index, philox.STREAM_J2,
                      pair_bounds=md.pair_bounds)
    vs[sample] -= (h * ACCEL / t.mass[sample])[:, None] * g0()
    md.v = vs
    md.step_index += 1


def cpu_baseline(s, steps=3, every=8):
    """The FP64 oracle as it stands, single-threaded numpy, on a bounded
    sample: `steps` BOUNCE steps of every `every`-th atom; time scaled."""
    from oracle.integrate import OracleMD
    topo, p = _oracle_setup(s)
    md = OracleMD(s.q, s.v, topo, p, seed=7, skin=SKIN, pair_bounds=True)
    sample = np.arange(0, s.n_atoms, every)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_sample_step(md, sample)
    dt = (time.perf_counter() - t0) * every / steps
    return {"value": round(ns_per_day(1, dt), 8), "unit": "ns/day", "cores": 1, "kind": "oracle",
            "sample": "%d BOUNCE steps of every %dth atom (%d atoms) of the 12288-atom droplet; time x%d" % (
                steps, every, len(sample), every)}


def reference_arm(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from paper_2002_07109_gb300.water import water_droplet
    from oracle.integrate import OracleMD
    s = water_droplet(N_SIDE, seed=0)
    topo, p = _oracle_setup(s)
    md = OracleMD(s.q, s.v, topo, p, seed=7, skin=SKIN, pair_bounds=True)
    every = 8
    sample = np.arange(0, s.n_atoms, every)
    for _ in range(args.warmup):
        oracle_sample_step(md, sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(md, sample)
    dt = (time.perf_counter() - t0) * every
    val = ns_per_day(args.steps, dt)
    sample_txt = "each step: BOUNCE on every %dth atom (%d of %d atoms); time x%d" % (every, len(sample), s.n_atoms,
                                                                                      every)
    print(json.dumps({
        "impl": "reference", "metric": "ns/day & pair-evals/s, BOUNCE vs BAOAB 1fs on one GB300 at matched <E>, RDF",
        "value": round(val, 8), "unit": "ns/day", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic: seeded lattice water droplet",
        "config": {"workload": "BOUNCE (per-type-pair bounds), 4096-molecule flexible-water droplet (12288 atoms), r_c 12 A, "
                               "cell list, "
                               "switch 4-5 A, 1 fs, friction 1/ps", "atoms": s.n_atoms},
        "cpu_baseline": {"value": round(val, 8), "unit": "ns/day", "cores": 1, "kind": "oracle", "sample": sample_txt},
        "e2e": {"value": round(val, 8), "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
