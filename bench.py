"""Benchmark: BOUNCE vs BAOAB (1 fs) on one GB300, at matched observables.

Headline workload: the periodic box of 32,768 flexible 3-site water
molecules (98,304 atoms, edge 99.3 A): Ewald direct erfc (beta 0.35 A^-1)
and Lennard-Jones within 9 A, SPME 96^3 of order 5, the Lennard-Jones part
beyond a 7.5-8.5 A switch on the jumps (Coulomb wholly in F_0, the split of
the paper's first example, Sec. IV.A), 1 fs, friction 1/ps.  `value` is
BOUNCE-RESPA (the reciprocal part on a 2 fs outer step, paper Sec. V) in
ns/day; `baoab` is BAOAB 1 fs on the same GPU; BOUNCE-RESPA1, plain BOUNCE
and BOUNCE-RESPA with Coulomb on the jumps too ride along.  One "step" is one 1 fs step
of the whole path (row and cluster rebuild checks, pair sums, SPME where the
integrator evaluates it, the jump half-steps, B, A, O).

Protocol (our arm):
  * the box is melted from the lattice with BAOAB (friction 0.05/fs, 2 ps)
    and relaxed at 1/ps (20 ps; the potential energy is flat over the last
    8 ps), all on the GPU;
  * each arm: W warm-up steps, then the K timed steps (rounded up to whole
    outer steps) in windows of 24 steps, one run() call each, with a 256 MB
    write before each window (L2 flushed); the trajectory continues across
    windows, so row and cluster rebuilds are inside the timed region;
  * device time by CUDA events on the launch stream; nvidia-smi clocks
    sampled during the timed windows;
  * e2e: the same windows through the public API with host arrays (state
    upload from host memory, run, state download), host wall clock;
  * per-kernel breakdown and the roofline of the pair kernel (the dominant
    kernel) from CUDA events around each group of launches
    (bounce_profile_breakdown) over 24 steps of the same trajectory;
  * matched observables: twelve independent runs per arm (own Philox seeds)
    from the relaxed box, 1.2 ps each to decorrelate, then 4.8 ps sampled every
    0.24 ps: potential energy per molecule, kinetic temperature, O-O g(r) and
    O self-diffusion; standard errors from the spread of the twelve runs; a
    second BAOAB arm with other seeds is the null control, BAOAB at 0.5 fs
    shows the comparator's own step-size error, and BOUNCE-RESPA without
    jumps (switch at the cutoff) separates the RESPA split from the jumps;
  * context: the 4,096-molecule droplet (r_c 12 A) with LJ on the jumps, the
    force-matching forward + backward on a 4,096-molecule box, and 256
    replica droplets of 64-1,024 molecules advanced together for 10,000 steps;
  * cpu_baseline: the FP64 oracle as it stands on a bounded sample of the
    workload (the same integrator on the 4,096-molecule box of the same
    density, cutoffs and grid spacing), on one core and on every core (one
    independent copy per core), scaled by the atom ratio.
--impl reference times the oracle alone (one core), each step one step of a
512-molecule box of the same density (the run ends within minutes).
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

METRIC = "ns/day & pair-evals/s, BOUNCE vs BAOAB 1fs on one GB300 at matched <E>, RDF"
WINDOW = 24        # steps per timed window (a multiple of every arm's outer step)
BOX_SIDE = 32      # 32^3 = 32,768 molecules
R_CUT, R_ON, R_OFF, SKIN, BETA, GRID, ORDER = 9.0, 7.5, 8.5, 1.0, 0.35, 96, 5
PAIR_SKIN = 3.0
DT = 1.0
RHO_O = 0.03343    # O atoms per A^3 at 1 g/cm^3
WORKLOAD = ("BOUNCE-RESPA (SPME on the 2 fs outer step) vs BAOAB 1 fs, 32,768-molecule periodic flexible-water box "
            "(98,304 atoms, edge 99.3 A), Ewald erfc beta 0.35 + LJ within 9 A, SPME 96^3 order 5, "
            "LJ beyond a 7.5-8.5 A switch on the jumps (Coulomb in F_0), 1 fs, friction 1/ps")
# Algorithmic lane-operations of one pair inside the cutoff in the cluster
# pair kernel, counted from the source: displacement 9, r^2 3, 1/r with a
# Newton step 5, r and 1/r^2 2, Ewald erfc term (A&S 7.1.26 and its
# exponential) 22, LJ 6, both sides' accumulation 6, charge product 2; the
# F_0 share adds the switching function and its weight (11).
OPS_PER_PAIR = {"f0": 66, "full": 55}
# DRAM traffic of one launch of the F_0 pair kernel on this machine (ncu
# dram__bytes_read.sum + dram__bytes_write.sum of k_cl_pairs<3>, the
# BOUNCE-RESPA part of `bench.py --profile box --steps 8`; cold caches)
PAIR_TRAFFIC = 24.08e6 + 2.6e3


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


def _reduce(x, ws, device, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def ns_per_day(steps, seconds):
    return steps * DT * 1e-6 * 86400.0 / seconds


def box_cfg(device, **kw):
    # cluster lists with a 3 A skin (rebuilt rarely; the pair kernel reads
    # lists pruned to r_c + 0.5 A every few steps)
    cfg = dict(r_on=R_ON, r_off=R_OFF, r_cut=R_CUT, skin=SKIN, pair_skin=PAIR_SKIN, dt=DT, ewald_beta=BETA,
               pme_grid=(GRID,) * 3, pme_order=ORDER, max_neighbors=1024, device=device)
    cfg.update(kw)
    return cfg


# The jump step's candidate rows are rebuilt when an atom has moved half
# their skin; a wider skin makes them rarer (and longer).  BAOAB reads no
# rows.
JUMP_ROWS = dict(skin=2.5, max_neighbors=2048)
# The headline split: LJ beyond the switch on the jumps, Coulomb in F_0
# (reading of the paper's first example).  With Coulomb on the jumps too the
# reflections heat flexible water at 1 fs (measured in matched_observables).
LJ_JUMPS = dict(JUMP_ROWS, jump_coulomb=False)
# (name, integrator name, extra config, outer period in steps)
BOX_ARMS = (("bounce_respa", "BOUNCE_RESPA", dict(LJ_JUMPS, respa_m=2), 2),
            ("baoab", "BAOAB", {}, 1),
            ("bounce_respa1", "BOUNCE_RESPA1", dict(LJ_JUMPS, respa_m=2, respa_m2=3), 6),
            ("bounce", "BOUNCE", dict(LJ_JUMPS), 1),
            ("bounce_respa_coulomb_jumps", "BOUNCE_RESPA", dict(JUMP_ROWS, respa_m=2), 2))


EQ_STRONG, EQ_STEPS, EQ_EVERY = 2000, 20000, 2000


def equilibrate_box(bounce, s, device, sh, seed):
    """Lattice -> liquid: BAOAB at friction 0.05/fs for 2 ps, then at the
    workload's 1/ps for 20 ps; returns the state and the trace of the
    temperature and the potential energy per molecule every 2 ps of the
    second part (flat over its last 8 ps when the box is relaxed)."""
    eq = bounce.from_system(s, seed=seed, gamma=0.05, **box_cfg(device))
    eq.set_state(s.q, s.v)
    eq.run(EQ_STRONG, bounce.BAOAB, stream=sh)
    q, v = eq.get_state(stream=sh)
    eq.close()
    eq = bounce.from_system(s, seed=seed + 1, **box_cfg(device))
    eq.set_state(q, v)
    n_mol = s.n_atoms // 3
    trace = []
    for _ in range(EQ_STEPS // EQ_EVERY):
        eq.run(EQ_EVERY, bounce.BAOAB, stream=sh)
        e = eq.energies(stream=sh)
        trace.append((round(e["temperature"], 1), round(e["potential"] / n_mol, 4)))
    q, v = eq.get_state(stream=sh)
    eq.close()
    return q, v, trace


def _round_up(k, m):
    return ((k + m - 1) // m) * m


def time_arm(bounce, ctx, q0, v0, integ, period, args, flush, stream, sh, ws, local, e2e=False):
    """W warm-up steps, then K timed steps (rounded up to whole outer steps)
    in windows (L2 flushed before each); the trajectory continues."""
    import torch
    steps = _round_up(args.steps, period)
    windows = [WINDOW] * (steps // WINDOW) + ([steps % WINDOW] if steps % WINDOW else [])
    ctx.set_state(q0, v0, step=0)
    ctx.run(_round_up(args.warmup, period), integ, stream=sh)
    torch.cuda.synchronize()
    ctx.reset_counters(stream=sh)
    ms, launches = 0.0, 0
    with Clocks(local) as clk:
        _barrier(ws)
        torch.cuda.synchronize()
        clk.start()
        for k, w in enumerate(windows):
            launches += ctx.run_launch_count(w, integ)
            flush.fill_(float(k))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.run(w, integ, stream=sh)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        torch.cuda.synchronize()
        clk.stop()
        _barrier(ws)
    out = dict(ms=ms, steps=steps, clocks=clk.summary(), energies=ctx.energies(stream=sh), launches=launches,
               windows=len(windows))
    if e2e:
        # the same windows through the public API with host buffers: state
        # upload from host memory, run, state download (the trajectory
        # continues through the host)
        q, v = ctx.get_state(stream=sh)
        step, t_e2e = 0, 0.0
        for w in windows:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_state(q, v, step=step)
            ctx.run(w, integ, stream=sh)
            q, v = ctx.get_state(stream=sh)
            t_e2e += time.perf_counter() - t0
            step += w
        out["e2e_s"] = t_e2e
        out["e2e_bytes"] = 2 * q.size * 8
    # per-kernel breakdown over 24 steps of the same trajectory
    ctx.reset_counters(stream=sh)
    ms_k, groups = ctx.profile_breakdown(WINDOW, integ, stream=sh)
    e = ctx.energies(stream=sh)
    out["breakdown"] = {k: round(v / WINDOW, 5) for k, v in ms_k.items()}
    out["pair_launch_ms"] = ms_k["pairs"] / max(int(groups[0]), 1)
    out["pairs_per_launch"] = (e["short_pairs"] + e["full_pairs"]) / max(int(groups[0]), 1)
    return out


def our_arm(args):
    import torch
    from paper_2002_07109_gb300 import bounce
    from paper_2002_07109_gb300.water import water_box

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    stream = torch.cuda.current_stream(device)
    sh = stream.cuda_stream
    s = water_box(BOX_SIDE, seed=rank)
    q0, v0, eq_trace = equilibrate_box(bounce, s, local, sh, 500 + rank)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)  # 256 MB > L2
    res = {}
    for name, integ, extra, period in BOX_ARMS:
        ctx = bounce.from_system(s, seed=21 + rank, **box_cfg(local, **extra))
        res[name] = time_arm(bounce, ctx, q0, v0, getattr(bounce, integ), period, args, flush, stream, sh, ws, local,
                             e2e=name == "bounce_respa")
        ctx.close()
    h, a = res["bounce_respa"], res["baoab"]
    t_h = _reduce(h["ms"] / 1e3, ws, device, "max")
    t_a = _reduce(a["ms"] / 1e3, ws, device, "max")
    value = ws * ns_per_day(h["steps"], t_h)
    baoab_value = ws * ns_per_day(a["steps"], t_a)
    n_atoms = s.n_atoms
    # pair evaluations per second: F_0 pairs + proposals (BOUNCE), full pairs (BAOAB)
    pe_h = _reduce(h["energies"]["short_pairs"] + h["energies"]["proposals"], ws, device, "sum") / t_h
    pe_a = _reduce(a["energies"]["full_pairs"], ws, device, "sum") / t_a
    clk = h["clocks"]
    sm_mhz = clk.get("sm_mhz") or 1995.0
    peak = 152 * 128 * sm_mhz * 1e6 / 1e12   # FP32/INT32 lane-ops per second at the sampled clock

    def roof(r, kind):
        return r["pairs_per_launch"] * OPS_PER_PAIR[kind] / (r["pair_launch_ms"] / 1e3) / 1e12

    ach = roof(h, "f0")
    e2e_val = ws * ns_per_day(h["steps"], _reduce(h["e2e_s"], ws, device, "max"))
    arms = {}
    for name, _, _, _ in BOX_ARMS:
        r = res[name]
        t = _reduce(r["ms"] / 1e3, ws, device, "max")
        e = r["energies"]
        arms[name] = {"value": round(ws * ns_per_day(r["steps"], t), 3), "unit": "ns/day",
                      "ms_per_step": round(t * 1e3 / r["steps"], 5), "steps": r["steps"],
                      "proposals_per_atom_step": round(e["proposals"] / (r["steps"] * n_atoms), 5),
                      "accepts_per_atom_step": round(e["accepts"] / (r["steps"] * n_atoms), 6),
                      "breakdown_ms_per_step": r["breakdown"],
                      "pair_kernel_ms_per_launch": round(r["pair_launch_ms"], 5),
                      "pairs_in_cutoff_per_launch": int(r["pairs_per_launch"]),
                      "temperature_end_K": round(e["temperature"], 1)}
    line = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "ns/day",
        "n_gpus": ws,
        "steps": h["steps"],
        "warmup": _round_up(args.warmup, 2),
        "ms_per_step": round(t_h * 1e3 / h["steps"], 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 pair math, f64 integration",
        "data": "synthetic: seeded lattice water box, melted and relaxed with BAOAB on the GPU",
        "config": {"workload": WORKLOAD, "atoms": n_atoms, "windows_of_steps": WINDOW,
                   "l2": "flushed before each timed window (256 MB write)",
                   "trajectory": "continues across windows (row, cluster and SPME work timed)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "baoab": {"value": round(baoab_value, 4), "unit": "ns/day", "ms_per_step": round(t_a * 1e3 / a["steps"], 5),
                  "pair_evals_per_s": pe_a},
        "speedup_vs_own_baoab": round(value / baoab_value, 4),
        "bounce_pair_evals_per_s": pe_h,
        "arms": arms,
        "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 3), "unit": "Tops/s",
                     "frac": round(ach / peak, 4), "traffic": PAIR_TRAFFIC,
                     "kernel": "k_cl_pairs (F_0 pair sums over the cluster lists, BOUNCE-RESPA)",
                     "algorithmic_ops": "%d lane-ops per unique pair inside r_c" % OPS_PER_PAIR["f0"],
                     "peak_source": "152 SMs x 128 FP32/INT32 lanes x sampled SM clock",
                     "baoab_pair_kernel_frac": round(roof(a, "full") / peak, 4)},
        "e2e": {"value": round(e2e_val, 4), "unit": "ns/day",
                "h2d_bytes_per_step": h["e2e_bytes"] * h["windows"] // h["steps"],
                "d2h_bytes_per_step": h["e2e_bytes"] * h["windows"] // h["steps"]},
        "gpu_launches": h["launches"],
        "clocks": clk,
    }
    line["matched_observables"] = matched_observables(bounce, s, q0, v0, local, stream, sh, rank)
    line["matched_observables"]["equilibration"] = {
        "protocol": "BAOAB %d steps at friction 0.05/fs, then %d steps at 1/ps" % (EQ_STRONG, EQ_STEPS),
        "T_K_and_Epot_per_molecule_every_2ps": eq_trace}
    line["droplet_context"] = droplet_context(bounce, local, stream, sh, rank, args)
    line["force_matching"] = force_matching(bounce, local, rank)
    line["batched_replicas"] = batched_replicas(bounce, local, stream, sh, rank)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _mean_se(x):
    x = np.asarray(x, dtype=np.float64)
    return x.mean(0), x.std(0, ddof=1) / math.sqrt(len(x))


def _welch(a, b):
    """Welch's comparison of two sets of run means (elementwise over the last
    axes): |t| = |mean_a - mean_b| / sqrt(se_a^2 + se_b^2), the
    Welch-Satterthwaite degrees of freedom, and the two-sided p-value from
    Student's t."""
    from scipy import stats
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ma, sa = _mean_se(a)
    mb, sb = _mean_se(b)
    va, vb = sa * sa, sb * sb
    den = np.sqrt(va + vb)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(den > 0, np.abs(ma - mb) / den, 0.0)
        nu = np.where(den > 0, (va + vb) ** 2 / (va * va / (len(a) - 1) + vb * vb / (len(b) - 1)), np.inf)
    return t, nu, 2.0 * stats.t.sf(t, nu)


def compare_arms(cur, ref, alpha=0.05, g_min=0.1):
    """An arm's run means against the reference arm's: potential energy,
    temperature and diffusion coefficient by Welch's test each, and g(r) over
    the bins where both arms reach g >= g_min (nearly empty bins get
    spuriously small errors from a few runs) by the largest per-bin Welch
    test, Bonferroni-corrected over those bins.  "matched": every one of the
    four p-values above alpha / 4 (a family-wise level alpha under the null).
    z is the Welch |t| of each scalar; chi^2 per bin and the largest bin |t|
    describe g(r)."""
    z, pv = {}, {}
    for k in ("pe", "T", "D"):
        t, _, pk = _welch(cur[k], ref[k])
        z[k] = round(float(t), 2)
        pv[k] = float(pk)
    gc = np.asarray(cur["g"], dtype=np.float64)
    gr = np.asarray(ref["g"], dtype=np.float64)
    keep = np.minimum(gc.mean(0), gr.mean(0)) >= g_min
    t, _, pb = _welch(gc[:, keep], gr[:, keep])
    nb = int(keep.sum())
    z["g_oo_chi2_per_bin"] = round(float((t ** 2).mean()), 2) if nb else 0.0
    z["g_oo_max_bin_z"] = round(float(t.max()), 2) if nb else 0.0
    z["g_oo_bins"] = nb
    pv["g"] = float(min(1.0, nb * pb.min())) if nb else 1.0
    z["p"] = {k: round(v, 4) for k, v in pv.items()}
    z["matched"] = bool(min(pv.values()) > alpha / 4)
    return z


def matched_observables(bounce, s, q0, v0, device, stream, sh, rank, runs=12, decor=1200, prod=4800, every=240):
    """Twelve independent runs per arm from the relaxed box (own Philox
    seeds, distinct between arms): `decor` steps, then `prod` steps sampled
    every `every` steps (all multiples of every arm's outer step).  Twelve
    runs, so that the standard errors taken from the spread of the runs are
    themselves stable.
    Per run: mean potential energy per molecule, mean kinetic temperature,
    O-O pair-distance histogram (0-8 A, 0.1 A bins) as g(r), and the O
    self-diffusion D from the mean squared displacement over the production
    (MSD(end) - MSD(middle)) / (6 * half the production).  Across runs: mean
    and standard error of the run means, compared with the BAOAB arm by
    compare_arms (Welch's tests, family-wise 5 %).  baoab_control is BAOAB
    with other seeds: the null."""
    import torch
    n_mol = s.n_atoms // 3
    n_o = int((s.type == 0).sum())
    L = float(s.box[0])
    edges = np.arange(81) * 0.1
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    # (name, integrator, extra config, outer period, seed base); dt from the config
    # every arm draws its own Philox streams (seed bases 1,000 apart): arms
    # that shared BAOAB's O-step noise would be correlated with it, and the
    # unpaired comparison would then understate their differences
    arms = (("baoab", "BAOAB", {}, 1, 1000),
            ("baoab_control", "BAOAB", {}, 1, 2000),
            ("baoab_half_fs", "BAOAB", dict(dt=0.5), 1, 3000),
            ("bounce_respa", "BOUNCE_RESPA", dict(LJ_JUMPS, respa_m=2), 2, 4000),
            ("bounce_respa1", "BOUNCE_RESPA1", dict(LJ_JUMPS, respa_m=2, respa_m2=3), 6, 5000),
            ("bounce_respa_no_jumps", "BOUNCE_RESPA", dict(LJ_JUMPS, respa_m=2, r_on=R_CUT, r_off=R_CUT), 2, 6000),
            ("bounce_respa_coulomb_jumps", "BOUNCE_RESPA", dict(JUMP_ROWS, respa_m=2), 2, 7000))
    raw = {}
    out = {"protocol": "%d runs per arm from the relaxed box, %d steps to decorrelate, then %d steps sampled every %d; "
                       "standard errors from the spread of the runs" % (runs, decor, prod, every)}
    for name, integ_name, extra, period, seed0 in arms:
        integ = getattr(bounce, integ_name)
        dt = extra.get("dt", DT)
        k_dt = int(round(DT / dt))      # steps per DT of simulated time
        per_run = {"pe": [], "T": [], "D": [], "g": []}
        ms, err = 0.0, None
        for r in range(runs):
            ctx = bounce.from_system(s, seed=seed0 + 17 * r + 100000 * rank, **box_cfg(device, **extra))
            try:
                ctx.set_state(q0, v0, step=0)
                ctx.run(decor * k_dt, integ, stream=sh)
                ctx.set_msd_reference(stream=sh)
                pe, T, hist, msd = [], [], np.zeros(80), {}
                for k in range(prod // every):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    ctx.run(every * k_dt, integ, stream=sh)
                    b.record(stream)
                    b.synchronize()
                    ms += a.elapsed_time(b)
                    e = ctx.energies(stream=sh)
                    pe.append((e["potential"]) / n_mol)
                    T.append(e["temperature"])
                    hist += ctx.pair_histogram(0, 0, 8.0, 80, stream=sh)
                    if k + 1 in (prod // every // 2, prod // every):
                        msd[k + 1] = ctx.msd(0, stream=sh)
                nk = prod // every
                per_run["pe"].append(np.mean(pe))
                per_run["T"].append(np.mean(T))
                per_run["g"].append(hist / nk * 2.0 / n_o / (RHO_O * shell))
                per_run["D"].append((msd[nk] - msd[nk // 2]) / (6.0 * (prod / 2) * DT / 1000.0))  # A^2/ps
            except Exception as ex:  # a blown-up state is reported, not compared
                err = str(ex).split("(")[0].strip()
            ctx.close()
            if err:
                break
        raw[name] = per_run
        res = {"runs": len(per_run["pe"])}
        if err:
            res["stopped"] = err
        if per_run["pe"]:
            res["ns_per_day"] = round(ns_per_day(len(per_run["pe"]) * prod, ms / 1e3), 2)   # simulated time
        if len(per_run["pe"]) >= 2:
            for k, unit in (("pe", "kcal/mol per molecule"), ("T", "K"), ("D", "A^2/ps")):
                m, se = _mean_se(per_run[k])
                res[k] = {"mean": round(float(m), 5), "se": round(float(se), 5), "unit": unit}
            m, _ = _mean_se(per_run["g"])
            kk = int(np.argmax(m[:40]))
            res["g_oo_first_peak"] = {"g": round(float(m[kk]), 4), "r_A": round(0.1 * (kk + 0.5), 2)}
            ref = raw.get("baoab")
            if name != "baoab" and ref and len(ref["pe"]) >= 2:
                res["z_vs_baoab"] = compare_arms(per_run, ref)
        out[name] = res
    # each arm's offset from BAOAB at 0.5 fs (the comparator's own step-size
    # error is BAOAB 1 fs's offset)
    half = raw.get("baoab_half_fs")
    if half and len(half["pe"]) >= 2:
        for name in out:
            if isinstance(out[name], dict) and name != "baoab_half_fs" and len(raw.get(name, {}).get("pe", [])) >= 2:
                d = {}
                for k in ("pe", "T"):
                    m1, e1 = _mean_se(raw[name][k])
                    m2, e2 = _mean_se(half[k])
                    d[k] = {"diff": round(float(m1 - m2), 5), "se": round(float(math.hypot(e1, e2)), 5)}
                out[name]["vs_baoab_half_fs"] = d
    return out


def droplet_context(bounce, device, stream, sh, rank, args):
    """The 4,096-molecule droplet (12,288 atoms, r_c 12 A): BOUNCE with LJ
    beyond the 4-5 A switch on the jumps (Coulomb in F_0) and BAOAB, K steps
    each in windows of 24 after W warm-up steps (context: the paper's droplet
    split with Coulomb on the jumps heats flexible water at 1 fs)."""
    import torch
    from paper_2002_07109_gb300.water import water_droplet
    s = water_droplet(16, seed=rank)
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=12.0, skin=1.0, dt=DT, device=device)
    eq = bounce.from_system(s, seed=1000 + rank, gamma=0.05, **cfg)
    eq.set_state(s.q, s.v)
    eq.run(1500, bounce.BAOAB, stream=sh)
    q0, v0 = eq.get_state(stream=sh)
    eq.close()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=torch.device("cuda", device))
    out = {"workload": "4,096-molecule flexible-water droplet (12,288 atoms), r_c 12 A, switch 4-5 A, 1 fs"}
    for name, integ, extra in (("bounce_lj_jumps", bounce.BOUNCE, dict(jump_coulomb=False)),
                               ("baoab", bounce.BAOAB, {})):
        ctx = bounce.from_system(s, seed=7 + rank, **cfg, **extra)
        r = time_arm(bounce, ctx, q0, v0, integ, 1, args, flush, stream, sh, 1, device)
        ctx.close()
        out[name] = {"value": round(ns_per_day(r["steps"], r["ms"] / 1e3), 2), "unit": "ns/day",
                     "breakdown_ms_per_step": r["breakdown"],
                     "temperature_end_K": round(r["energies"]["temperature"], 1)}
    return out


def batched_replicas(bounce, device, stream, sh, rank, n_steps=10000, n_baoab=1000):
    """256 independent droplets of 64-1,024 molecules (seeded sizes), each
    with its own Philox seed, in one context: every step advances every
    replica in the same launches; run() replays one CUDA graph per 32 steps;
    the all-pairs pair kernel is a resident grid over the static work queue
    of (replica, 32-atom i-tile, j-block) items, its j-block length and grid
    chosen by the autotuner.  BOUNCE with LJ beyond the 4-5 A switch on the
    jumps (Coulomb in F_0), and BAOAB beside it; aggregate ns/day (sum over
    replicas) and replica-steps per second."""
    import torch
    from paper_2002_07109_gb300.water import concat_systems, replica_sizes, water_droplet_molecules
    sizes = replica_sizes(256, seed=rank)
    systems = [water_droplet_molecules(int(m), seed=100 + r + 1000 * rank) for r, m in enumerate(sizes)]
    cat, off = concat_systems(systems)
    seeds = np.arange(256, dtype=np.uint64) + 7 + 1000 * rank
    out = {"workload": "256 droplets of 64-1,024 molecules (%d atoms in all), no cutoff, switch 4-5 A, 1 fs"
                       % cat.n_atoms}
    stream = torch.cuda.current_stream(torch.device("cuda", device))
    cfg = dict(r_on=4.0, r_off=5.0, r_cut=math.inf, jump_coulomb=False, max_neighbors=int(np.diff(off).max()),
               device=device)
    # the lattice droplets melted with BAOAB at friction 0.05/fs (2 ps), both arms from there
    eq = bounce.from_system(cat, seed=1, gamma=0.05, **cfg)
    eq.set_replicas(off, seeds)
    eq.set_state(cat.q, cat.v)
    eq.run(2000, bounce.BAOAB, stream=sh)
    q0, v0 = eq.get_state(stream=sh)
    eq.close()
    out["start"] = "BAOAB at friction 0.05/fs for 2 ps from the lattice droplets"
    for name, integ, steps in (("bounce_lj_jumps", bounce.BOUNCE, n_steps), ("baoab", bounce.BAOAB, n_baoab)):
        ctx = bounce.from_system(cat, seed=1, **cfg)
        ctx.set_replicas(off, seeds)
        ctx.set_state(q0, v0)
        tune = ctx.autotune(integ, stream=sh)
        ctx.run(64, integ, stream=sh)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.run(steps, integ, stream=sh)
        b.record(stream)
        b.synchronize()
        sec = a.elapsed_time(b) / 1e3
        e = ctx.energies(stream=sh)
        ctx.close()
        # the tile pair kernel's roofline: every pair of different molecules
        # of each replica once, at the algorithmic lane-operations per pair
        n_pairs = float(sum(9 * int(m) * (int(m) - 1) // 2 for m in sizes))
        ops = OPS_PER_PAIR["f0" if integ != bounce.BAOAB else "full"]
        ach = n_pairs * ops / (tune["pair_ms"] / 1e3) / 1e12
        peak = 152 * 128 * 2070e6 / 1e12
        out[name] = {"steps": steps, "aggregate_ns_per_day": round(256 * ns_per_day(steps, sec), 2),
                     "replica_steps_per_s": round(256 * steps / sec, 1), "ms_per_step": round(sec * 1e3 / steps, 4),
                     "tuning": {"tile_j": tune["tile_j"], "tile_blocks": tune["tile_blocks"],
                                "pair_kernel_ms": round(tune["pair_ms"], 4)},
                     "pair_kernel_roofline": {"bound": "alu", "pairs_per_launch": n_pairs, "achieved": round(ach, 3),
                                              "peak": round(peak, 3), "unit": "Tops/s", "frac": round(ach / peak, 4),
                                              "peak_source": "152 SMs x 128 lanes x 2,070 MHz (max SM clock)"},
                     "temperature_end_K": round(e["temperature"], 1)}
    return out


def force_matching(bounce, device, rank, reps=5):
    """Forward + backward of the force-matching loss sum |F - F_t|^2 through
    the autograd binding on the 4,096-molecule box (Ewald erfc beta 0.35 and
    LJ within 9 A); time per evaluation (CUDA events)."""
    import torch
    from paper_2002_07109_gb300.water import water_box
    s = water_box(16, seed=7 + rank)
    dev = torch.device("cuda", device)
    ctx = bounce.from_system(s, seed=1, r_on=4.0, r_off=5.0, r_cut=9.0, ewald_beta=BETA, skin=1.0,
                             max_neighbors=1024, device=device)
    ctx.set_state(s.q, s.v)
    qt = torch.tensor([-0.834, 0.417], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor([[3.15, 0.0], [0.0, 0.0]], dtype=torch.float64, requires_grad=True)
    eps = torch.tensor([[0.152, 0.0], [0.0, 0.0]], dtype=torch.float64, requires_grad=True)
    q = torch.tensor(s.q, dtype=torch.float64, device=dev, requires_grad=True)
    Fn = bounce.pair_forces_function()
    F_t = torch.zeros((s.n_atoms, 3), dtype=torch.float64, device=dev)
    ms = []
    for k in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        F, E = Fn.apply(q, qt, sig, eps, ctx)
        loss = ((F - F_t) ** 2).sum() + 0.5 * E.to(dev)
        loss.backward()
        b.record()
        b.synchronize()
        if k:
            ms.append(a.elapsed_time(b))
    ctx.close()
    return {"workload": "force matching, 4,096-molecule box (12,288 atoms), r_c 9 A", "ms_per_forward_backward":
            round(float(np.median(ms)), 3)}


def _oracle_sample(side=16):
    """A bounded sample of the workload: a box of side^3 molecules at the
    same density (side 16: 4,096 molecules, edge 49.7 A), the same cutoffs,
    switch and Ewald beta, an SPME grid of the same spacing (3 side), the
    BOUNCE-RESPA split of the workload."""
    from oracle.forcefield import Params
    from oracle.integrate import OracleMD, Topology
    from paper_2002_07109_gb300.water import water_box
    s = water_box(side, seed=0)
    topo = Topology(s.type, s.mass, s.charge, s.molecule, s.bonds, s.bond_k_r0, s.angles, s.angle_k_t0)
    p = Params(r_on=R_ON, r_off=R_OFF, r_cut=R_CUT, ewald_beta=BETA, box=s.box, lj_sigma=s.lj_sigma,
               lj_eps=s.lj_eps, pme_grid=(3 * side,) * 3, pme_order=ORDER)
    return OracleMD(s.q, s.v, topo, p, seed=7, skin=SKIN), s.n_atoms


def _oracle_blocks(n_blocks):
    """Worker: n_blocks BOUNCE-RESPA outer steps (2 steps each) of the
    oracle on the sample; returns the wall time."""
    md, _ = _oracle_sample()
    md.ensure_rows()
    t0 = time.perf_counter()
    for _ in range(n_blocks):
        md.block_bounce_respa(2)
    return time.perf_counter() - t0


def cpu_baseline(blocks=1):
    """The oracle on the sample: one core, then one independent copy per
    host core at once (spawned processes); ns/day of the full 98,304-atom
    workload, scaled by the atom ratio (98,304 / 12,288 = 8)."""
    import multiprocessing as mp
    scale = (BOX_SIDE ** 3 * 3) / (16 ** 3 * 3)
    t1 = _oracle_blocks(blocks)
    single = ns_per_day(2 * blocks, t1 * scale)
    cores = os.cpu_count() or 1
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            times = pool.map(_oracle_blocks, [blocks] * cores)
            wall = time.perf_counter() - t0
        allcore = cores * ns_per_day(2 * blocks, max(times) * scale)
    except Exception:
        allcore, wall = None, None
    return {"value": round(single, 8), "unit": "ns/day", "cores": 1, "kind": "oracle",
            "sample": "%d BOUNCE-RESPA steps of the oracle on the 4,096-molecule box of the workload's density, "
                      "cutoffs and grid spacing (12,288 atoms, 48^3), single-threaded numpy; time x %.0f (atom "
                      "ratio)" % (2 * blocks, scale),
            "all_cores": {"value": None if allcore is None else round(allcore, 8), "cores": cores,
                          "how": "one independent copy of the sample per core at once (aggregate throughput)",
                          "wall_s": None if wall is None else round(wall, 2)}}


REF_SIDE = 8   # the reference arm's sample: 512 molecules (1,536 atoms), ~0.5 s per oracle step


def reference_arm(args):
    """The oracle alone: each step one BOUNCE-RESPA step of the sample (the
    512-molecule box of the workload's density, edge 24.8 A, one core), so
    that the default run ends within a few minutes; ms_per_step is the
    measured sample step, value the ns/day of the 98,304-atom workload scaled
    by the atom ratio (the oracle's step is linear in the atoms: cell lists
    and an SPME grid of fixed spacing)."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    md, n_sample = _oracle_sample(REF_SIDE)
    md.ensure_rows()
    scale = (BOX_SIDE ** 3 * 3) / n_sample
    for _ in range(max(1, _round_up(args.warmup, 2) // 2)):
        md.block_bounce_respa(2)
    steps = _round_up(args.steps, 2)
    t0 = time.perf_counter()
    for _ in range(steps // 2):
        md.block_bounce_respa(2)
    dt = time.perf_counter() - t0
    val = ns_per_day(steps, dt * scale)
    sample = ("each step: one BOUNCE-RESPA step of the oracle on the %d-molecule box of the workload's density, "
              "cutoffs and grid spacing (%d atoms), single-threaded numpy; ns/day scaled by the atom ratio %.0f"
              % (n_sample // 3, n_sample, scale))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(val, 8), "unit": "ns/day", "n_gpus": ws,
        "steps": steps, "warmup": _round_up(args.warmup, 2), "ms_per_step": round(dt * 1e3 / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded lattice water box", "config": {"workload": WORKLOAD, "atoms": BOX_SIDE ** 3 * 3},
        "cpu_baseline": {"value": round(val, 8), "unit": "ns/day", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 8), "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def profile_case(args):
    """A few steps of one workload for profiler captures (no timing, no
    JSON line): box -- the 98,304-atom box, BAOAB then BOUNCE-RESPA from a
    short BAOAB relaxation; batch -- the 256 replica droplets, BOUNCE; droplet
    -- the 4,096-molecule droplet, BAOAB then BOUNCE (LJ on the jumps)."""
    import torch
    from paper_2002_07109_gb300 import bounce
    from paper_2002_07109_gb300.water import concat_systems, replica_sizes, water_box, water_droplet, \
        water_droplet_molecules
    n = _round_up(max(args.steps, 2), 2)
    if args.profile == "box":
        s = water_box(BOX_SIDE, seed=0)
        eq = bounce.from_system(s, seed=500, gamma=0.05, **box_cfg(0))
        eq.set_state(s.q, s.v)
        eq.run(48, bounce.BAOAB)
        q, v = eq.get_state()
        eq.close()
        for integ, extra in ((bounce.BAOAB, {}), (bounce.BOUNCE_RESPA, dict(LJ_JUMPS, respa_m=2))):
            ctx = bounce.from_system(s, seed=21, **box_cfg(0, **extra))
            ctx.set_state(q, v)
            ctx.run(n, integ)
            torch.cuda.synchronize()
            ctx.close()
    elif args.profile == "batch":
        sizes = replica_sizes(256, seed=0)
        cat, off = concat_systems([water_droplet_molecules(int(m), seed=100 + r) for r, m in enumerate(sizes)])
        ctx = bounce.from_system(cat, seed=1, r_on=4.0, r_off=5.0, r_cut=math.inf, jump_coulomb=False,
                                 max_neighbors=int(np.diff(off).max()))
        ctx.set_replicas(off, np.arange(256, dtype=np.uint64) + 7)
        ctx.set_state(cat.q, cat.v)
        ctx.run(n, bounce.BOUNCE)
        torch.cuda.synchronize()
        ctx.close()
    else:
        s = water_droplet(16, seed=0)
        cfg = dict(r_on=4.0, r_off=5.0, r_cut=12.0, skin=1.0)
        for integ, extra in ((bounce.BAOAB, {}), (bounce.BOUNCE, dict(jump_coulomb=False))):
            ctx = bounce.from_system(s, seed=7, **cfg, **extra)
            ctx.set_state(s.q, s.v)
            ctx.run(n, integ)
            torch.cuda.synchronize()
            ctx.close()
    print("profile case %s done" % args.profile)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", choices=["box", "batch", "droplet"], default=None,
                    help="run a few steps of one workload for a profiler capture and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile:
        profile_case(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
