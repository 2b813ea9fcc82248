"""Benchmark: BOUNCE vs BAOAB (1 fs) on a 4,096-molecule flexible-water
droplet (12,288 atoms, 12 A cutoff, cell list) on one GB300.

One "step" is one full integrator step (row-rebuild check, F_0 or the full
gradient, the two jump half-steps, B, A, O).  The headline value is BOUNCE
ns/day with the split that keeps the observables of BAOAB 1 fs: LJ beyond
the 4-5 A switch on the jumps, Coulomb in F_0.  BAOAB
ns/day, pair evaluations per second and the matched-observables comparison
ride along, with the paper's droplet split (Coulomb on the jumps too), which
heats flexible water at 1 fs.

Protocol (our arm):
  * the droplet is pre-equilibrated on the GPU with BAOAB (friction 0.05/fs,
    1,500 steps) from the seeded lattice;
  * W warm-up steps, then the K timed steps in windows of 25 steps (one
    run() call each); the trajectory continues across windows, so the row
    rebuilds it triggers are inside the timed region;
  * L2 is flushed (a 256 MB write) before each timed window;
  * device time by CUDA events on the launch stream; nvidia-smi clocks are
    sampled during the timed windows;
  * e2e: the same windows through the public API with host buffers (state
    upload, run, state download), host wall clock;
  * roofline: the fused step kernel timed by CUDA events around each launch
    in a separate profiling pass of the same workload;
  * the heating split runs 5-step windows, each restarted from the
    equilibrated state, and reports its temperature after each window;
  * matched observables: 100 ps per integrator (block means of the potential
    energy, temperature, O-O pair-distance histogram and O self-diffusion);
  * a periodic-box section (98,304 atoms, SPME) compares BAOAB with
    BOUNCE-RESPA and BOUNCE-RESPA1.
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

WINDOW = 25       # steps per timed window (one run() call); L2 flushed between windows
HOT_WINDOW = 5    # windows of the split that heats, each restarted from the 300 K state
# the headline split: LJ beyond the 4-5 A switch on the jumps, Coulomb (12 A
# cutoff) in F_0, one bound per atom type (with ~0.1 proposals per atom-step
# the two-stage choice of per-type-pair bounds saves less than its
# type-grouped rows cost in the row builds and the F_0 gathers)
SPLIT = dict(pair_bounds=False, jump_coulomb=False)
RHO_O = 0.03343   # O atoms per A^3 in water at 1 g/cm^3
# (name, integrator, split, restart every window)
ARMS = (("bounce", "BOUNCE", SPLIT, False),
        ("baoab", "BAOAB", {}, False),
        ("bounce_coulomb_jumps", "BOUNCE", dict(pair_bounds=True), True),
        ("bounce_coulomb_jumps_rowmax", "BOUNCE", dict(pair_bounds=False), True))
WORKLOAD = ("BOUNCE (LJ beyond the 4-5 A switch on jumps, Coulomb in F_0), "
            "4096-molecule flexible-water droplet (12288 atoms), r_c 12 A, cell list, 1 fs, friction 1/ps")
N_SIDE = 16                  # 16^3 = 4096 molecules
R_CUT, R_ON, R_OFF, SKIN = 12.0, 4.0, 5.0, 1.0
DT = 1.0
# DRAM bytes (read + write) of one body step (pair-sum kernel + step kernel)
# with this split on the same-size droplet at its lattice start (ncu, cold
# caches; ~670 row entries per atom there, ~920 after equilibration)
K_STEP_TRAFFIC = (34264320 + 768) + (2803200 + 0)  # k_pairs + k_step<BOUNCE>
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


def _windows(steps, w_len):
    return [w_len] * (steps // w_len) + ([steps % w_len] if steps % w_len else [])


def time_arm(bounce, s, q0, v0, cfg, integ, extra, restart, args, flush, stream, sh, ws, rank, local, name,
             e2e=False, profile=False):
    """K timed steps of one integrator in windows (L2 flushed before each);
    continuing arms carry the trajectory across windows, so the row rebuilds
    it triggers are timed; restarting arms begin every window at the
    equilibrated state (a split that heats)."""
    import torch
    w_len = HOT_WINDOW if restart else WINDOW
    windows = _windows(args.steps, w_len)
    ctx = bounce.from_system(s, seed=7 + rank, **cfg, **extra)
    ctx.set_state(q0, v0, step=0)
    ctx.run(args.warmup, integ, stream=sh)
    torch.cuda.synchronize()
    ctx.reset_counters(stream=sh)
    ms, launches, t_end = 0.0, 0, []
    with Clocks(local) as clk:
        _barrier(ws)
        torch.cuda.synchronize()
        clk.start()
        torch.cuda.nvtx.range_push(name + "_timed")
        for k, w in enumerate(windows):
            if restart:
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
            if restart:
                t_end.append(ctx.energies(stream=sh)["temperature"])
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clk.stop()
        _barrier(ws)
    e = ctx.energies(stream=sh)
    out = dict(ms=ms, clocks=clk.summary(), energies=e, t_end=t_end, launches=launches, windows=len(windows),
               w_len=w_len)
    if e2e:
        # the same windows through the public API with host buffers: state
        # upload, run, state download (the trajectory continues on the host)
        q, v, step, t_e2e = q0, v0, 200000, 0.0
        for k, w in enumerate(windows):
            if restart:
                q, v = q0, v0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_state(q, v, step=step)
            ctx.run(w, integ, stream=sh)
            q, v = ctx.get_state(stream=sh)
            t_e2e += time.perf_counter() - t0
            step += w
        out["e2e_s"] = t_e2e
    if profile:
        # fused step kernel timed by CUDA events around each launch
        ctx.set_state(q0, v0, step=300000)
        ctx.reset_counters(stream=sh)
        out["kernel_ms"], out["kernel_launches"] = ctx.profile_steps(min(args.steps, WINDOW), integ, stream=sh)
        out["prof"] = ctx.energies(stream=sh)
    ctx.close()
    return out


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
    res = {}
    for name, integ, extra, restart in ARMS:
        res[name] = time_arm(bounce, s, q0, v0, cfg, getattr(bounce, integ), extra, restart, args, flush, stream, sh,
                             ws, rank, local, name, e2e=name == "bounce", profile=name in ("bounce", "baoab"))
    steps = args.steps
    n_atoms = s.n_atoms
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
    ops_a = OPS_PER_FULL_PAIR * a["prof"]["full_pairs"]
    ach_a = ops_a / a["kernel_launches"] / (a["kernel_ms"] / 1e3 / a["kernel_launches"]) / 1e12
    h2d = 2 * n_atoms * 3 * 8
    e2e_val = ws * ns_per_day(steps, _max_over_ranks(b["e2e_s"], ws, device))

    def hot(name):
        r = res[name]
        t = _max_over_ranks(r["ms"] / 1e3, ws, device)
        e = r["energies"]
        return {"value": round(ws * ns_per_day(steps, t), 4), "unit": "ns/day",
                "proposals_per_atom_step": round(e["proposals"] / (steps * n_atoms), 3),
                "accepts_per_atom_step": round(e["accepts"] / (steps * n_atoms), 3),
                "temperature_end_of_windows_K": [round(x, 1) for x in r["t_end"]][:4]}

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
        "config": {"workload": WORKLOAD, "atoms": n_atoms, "windows_of_steps": WINDOW,
                   "l2": "flushed before each timed window",
                   "trajectory": "continues across windows (row rebuilds are timed)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "baoab": {"value": round(baoab_value, 4), "unit": "ns/day", "ms_per_step": round(t_a * 1e3 / steps, 5),
                  "pair_evals_per_s": pe_a},
        "bounce_pair_evals_per_s": pe_b,
        "speedup_vs_own_baoab": round(value / baoab_value, 4),
        "proposals_per_atom_step": b["energies"]["proposals"] / (steps * n_atoms),
        "accepts_per_atom_step": b["energies"]["accepts"] / (steps * n_atoms),
        "near_ties": b["energies"]["near_ties"],
        "rebuilds_in_timed_region": {"bounce": b["energies"]["rebuilds"], "baoab": a["energies"]["rebuilds"]},
        "temperature_after_timed_steps_K": {"bounce": round(b["energies"]["temperature"], 1),
                                            "baoab": round(a["energies"]["temperature"], 1)},
        "bounce_coulomb_jumps": dict(
            hot("bounce_coulomb_jumps"),
            split="Coulomb and LJ beyond the 4-5 A switch on the jumps (the paper's droplet split); it heats "
                  "flexible water at 1 fs, so each %d-step window restarts from the 300 K state" % HOT_WINDOW,
            rowmax_bounds=hot("bounce_coulomb_jumps_rowmax")),
        "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 3), "unit": "Tops/s",
                     "frac": round(achieved / peak, 4), "traffic": K_STEP_TRAFFIC,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, the k_pairs and "
                                       "k_step<BOUNCE> launches of one body step with this split on the "
                                       "same-size lattice droplet",
                     "kernel": "k_pairs + k_step<BOUNCE> (F_0 pair sums; bonded terms, 2 jump half-steps, "
                               "B A O A)",
                     "baoab_kernel_frac": round(ach_a / peak, 4)},
        "e2e": {"value": round(e2e_val, 4), "unit": "ns/day", "h2d_bytes_per_step": h2d * b["windows"] // steps,
                "d2h_bytes_per_step": h2d * b["windows"] // steps},
        "gpu_launches": b["launches"],
        "clocks": clk,
    }
    line["matched_observables"] = matched_observables(s, q0, v0, cfg, rank, stream, sh)
    line["pbc_box"] = pbc_box(rank, stream, sh)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(s)
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _block_stats(x):
    x = np.asarray(x, dtype=np.float64)
    return x.mean(0), x.std(0, ddof=1) / math.sqrt(len(x))


def matched_observables(s, q0, v0, cfg, rank, stream, sh, n_eq=5000, n_blocks=50, block=2000, samples=10):
    """Long runs from the equilibrated droplet for the matched-observables
    comparison with BAOAB 1 fs: n_eq steps of equilibration, then n_blocks
    blocks of `block` steps (100 ps).  Per block: the means of the potential
    energy per molecule, the kinetic temperature and the O-O pair-distance
    histogram (0-8 A, 0.2 A bins, pairs per O atom; the droplet's RDF
    observable, reported as g(r) over bulk density) over `samples` evenly
    spaced samples, and the self-diffusion
    coefficient of O from the growth of the mean squared displacement between
    the block's middle and end (D = (MSD(2 ps) - MSD(1 ps)) / 6 ps).  Each arm
    is compared with BAOAB by z = |difference of block means| / combined
    standard error (RDF: chi^2 per bin over the bins with counts, and the
    largest per-bin z).  ns/day here are over graph-captured chunks without
    L2 flushes, for context."""
    import torch
    from paper_2002_07109_gb300 import bounce
    n_mol = s.n_atoms // 3
    n_o = int((s.type == 0).sum())
    # baoab_control: BAOAB again with other Philox streams, the null
    # comparison that shows the spread of z between two runs of one method
    arms = (("baoab", bounce.BAOAB, {}, 31),
            ("baoab_control", bounce.BAOAB, {}, 131),
            ("bounce", bounce.BOUNCE, SPLIT, 31),
            ("bounce_respa_ext_2fs", bounce.BOUNCE_RESPA_EXT, dict(SPLIT, respa_m=2), 31))
    chunk = block // samples
    edges = np.arange(41) * 0.2
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    raw, out = {}, {"protocol": "%d equilibration steps, then %d blocks of %d steps (%g ps) per arm, from the "
                                "BAOAB-equilibrated droplet; friction 1/ps" % (n_eq, n_blocks, block,
                                                                                n_blocks * block / 1000)}
    for name, integ, extra, seed in arms:
        ctx = bounce.from_system(s, seed=seed + rank, **cfg, **extra)
        ctx.set_state(q0, v0, step=0)
        obs = {"pe": [], "T": [], "D": [], "rdf": []}
        ms, err = 0.0, None
        try:
            ctx.run(n_eq, integ, stream=sh)
            for _ in range(n_blocks):
                ctx.set_msd_reference(stream=sh)
                pe, T, rdf, msd = [], [], np.zeros(40), []
                for k in range(samples):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ctx.run(chunk, integ, stream=sh)
                    b.record(stream)
                    b.synchronize()
                    ms += a.elapsed_time(b)
                    e = ctx.energies(stream=sh)
                    pe.append(e["potential"] / n_mol)
                    T.append(e["temperature"])
                    rdf += ctx.pair_histogram(0, 0, 8.0, 40, stream=sh) * (2.0 / n_o)
                    if k in (samples // 2 - 1, samples - 1):
                        msd.append(ctx.msd(0, stream=sh))
                obs["pe"].append(np.mean(pe))
                obs["T"].append(np.mean(T))
                obs["rdf"].append(rdf / samples)
                obs["D"].append((msd[1] - msd[0]) / (6.0 * block / 2000.0))  # A^2/ps
        except Exception as ex:  # a blown-up state is reported, not compared
            err = str(ex).split("(")[0].strip()
        ctx.close()
        raw[name] = obs
        r = {"steps": n_eq + len(obs["pe"]) * block}
        if err:
            r["stopped"] = err
        else:
            r["ns_per_day"] = round(ns_per_day(n_blocks * block, ms / 1e3), 2)
            for k, unit in (("pe", "kcal/mol per molecule"), ("T", "K"), ("D", "A^2/ps")):
                m, se = _block_stats(obs[k])
                r[k] = {"mean": round(float(m), 4), "se": round(float(se), 4), "unit": unit}
            m, _ = _block_stats(obs["rdf"])
            g = m / (RHO_O * shell)   # pairs per O over the bulk-water expectation: g(r) of the droplet
            k = int(np.argmax(g[:20]))
            r["rdf_oo_first_peak"] = {"g": round(float(g[k]), 4), "r_A": round(0.2 * (k + 0.5), 2)}
            if name != "baoab" and "rdf" in raw.get("baoab", {}) and raw["baoab"]["rdf"]:
                ref = raw["baoab"]
                z = {}
                for k in ("pe", "T", "D"):
                    m1, e1 = _block_stats(obs[k])
                    m2, e2 = _block_stats(ref[k])
                    z[k] = round(float(abs(m1 - m2) / math.hypot(e1, e2)), 2)
                m1, e1 = _block_stats(obs["rdf"])
                m2, e2 = _block_stats(ref["rdf"])
                ok = (e1 + e2) > 0
                zb = np.abs(m1 - m2)[ok] / np.hypot(e1, e2)[ok]
                z["rdf_chi2_per_bin"] = round(float((zb ** 2).mean()), 2)
                z["rdf_max_bin_z"] = round(float(zb.max()), 2)
                r["z_vs_baoab"] = z
        out[name] = r
    return out


def pbc_box(rank, stream, sh, n_steps=960, chunk=48):
    """The periodic box of 32,768 water molecules (98,304 atoms, edge 99.3 A):
    Ewald direct erfc (beta 0.35) and LJ within 9 A, SPME 96^3 of order 5,
    jumps beyond a 7.5-8.5 A switch (one bound per atom type), 1 fs, friction
    1/ps.  From a BAOAB-equilibrated state, graph-captured runs of n_steps
    after one warm-up chunk: BAOAB (SPME every step), BOUNCE (SPME every
    step), BOUNCE-RESPA (SPME on the 2 fs outer step) and BOUNCE-RESPA1
    (short-range pairs on 2 fs, SPME on 6 fs).  ns/day over the chunks (CUDA events), and the means of the
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
            ("bounce", bounce.BOUNCE, dict(pair_bounds=False)),
            ("bounce_respa", bounce.BOUNCE_RESPA, dict(pair_bounds=False, respa_m=2)),
            ("bounce_respa1", bounce.BOUNCE_RESPA1, dict(pair_bounds=False, respa_m=2, respa_m2=3)))
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
    p = Params(r_on=R_ON, r_off=R_OFF, r_cut=R_CUT, lj_sigma=s.lj_sigma, lj_eps=s.lj_eps,
               coulomb_jumps=SPLIT["jump_coulomb"])
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
    md = OracleMD(s.q, s.v, topo, p, seed=7, skin=SKIN, pair_bounds=SPLIT["pair_bounds"])
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
    md = OracleMD(s.q, s.v, topo, p, seed=7, skin=SKIN, pair_bounds=SPLIT["pair_bounds"])
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
        "config": {"workload": WORKLOAD, "atoms": s.n_atoms},
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
