"""Benchmark: checkerboard Metropolis sweeps of the 2D Ising model on GB300.

One step = one sweep (black half-sweep, then white half-sweep with the fused
{M, bond sum} reduction) of a multi-spin-coded 65536 x 65536 lattice (4.3e9
spins, two 1.07 GB colour planes: larger than L2, so no flush is needed),
random start from seed 1234, beta = 0.4406868.  The metric is spin flips/ns =
L^2 x sweeps / ns (attempted updates).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun and cuts the one lattice into N horizontal slabs,
one per GPU, with the boundary rows exchanged point to point (NCCL) beside
the interior updates (Sec. 4; strong scaling: the lattice is the same for
every N); ``--workload replicas`` runs one independent lattice per GPU
instead (weak scaling, seed 1234 + rank, no data-path collective).  The value
is all ranks' flips divided by the slowest rank's time.  ``--impl reference`` times the CPU oracle
(the plain C implementation the kernels are checked against) on the host
cores instead.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin flips/ns at 1 GB300 (% of roofline)"
UNIT = "flips/ns"
BETA_C_CONFIG = 0.4406868
PAPER_CONTEXT = "417.53 flips/ns, multi-spin code, (123x2048)^2, 1x V100-SXM (Table 2); other hardware"


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--L", type=int, default=65536)
    p.add_argument("--beta", type=float, default=BETA_C_CONFIG)
    p.add_argument("--seed", type=int, default=1234)
    p.add_argument("--init", choices=["random", "up"], default="random")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--cpu-L", type=int, default=16384, help="oracle sample lattice side")
    p.add_argument("--cpu-sweeps", type=int, default=20, help="oracle sample sweeps (all cores)")
    p.add_argument("--ref-L", type=int, default=8192, help="oracle lattice side of one reference-arm step")
    p.add_argument("--cpu-sweeps-1t", type=int, default=1, help="oracle sweeps of 16384^2 on one thread")
    p.add_argument("--cpu-short", action="store_true",
                   help="cpu baseline: only the headline sample (no 1-thread, 256^2 or 65536^2 spot check)")
    p.add_argument("--no-extras", action="store_true", help="skip per-beta, rng probe, e2e and cpu legs")
    p.add_argument("--no-batch", action="store_true", help="skip the batched parallel-tempering leg")
    p.add_argument("--pt-sweeps", type=int, default=10000)
    p.add_argument("--pt-ess-sweeps", type=int, default=100000,
                   help="sweeps of each matched-error run of the batch (with and without exchanges)")
    p.add_argument("--pt-ess-warm", type=int, default=20000, help="sweeps before the matched-error records")
    p.add_argument("--slabs", type=int, default=4, help="slabs on one GPU for the slab leg / workload")
    p.add_argument("--no-binder", action="store_true", help="skip the Binder-crossing leg")
    p.add_argument("--binder-sweeps", type=int, default=100000)
    p.add_argument("--workload", choices=["sweep", "replicas", "pt", "learned", "network", "train", "slabs", "binder",
                                          "host", "probes"],
                   default="sweep",
                   help="sweep: the 65536^2 lattice (default; with several GPUs cut into one slab per rank); "
                        "replicas: one independent lattice per GPU; pt / learned / ...: only that leg")
    p.add_argument("--no-learned", action="store_true", help="skip the learned block-proposal leg")
    p.add_argument("--learned-steps", type=int, default=1000, help="training steps of the proposal network")
    p.add_argument("--learned-cycles", type=int, default=32000,
                   help="measured sweep + move cycles (at least 50 tau_int of |m| at 128^2, beta_c)")
    p.add_argument("--learned-configs", type=int, default=100000, help="training configurations")
    p.add_argument("--learned-chains", type=int, default=1024, help="chains of the measured learned cycles")
    p.add_argument("--net-reps", type=int, default=10, help="timed network evaluations (--workload network)")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed plumbing (timing only; no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(base: int, rank: int) -> int:
    return base + rank


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ids = [x.strip() for x in vis.split(",")] if vis else []
        self.gpu = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.path is None:
            return None
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Integer roofline of the sweep kernel.  A spin update needs a quarter of a
# Philox4x32-10 block: 20 32x32->64-bit multiplies per 4 draws.  The peak rate
# of that multiply is measured by the wide-multiply probe (ising_mulwide_probe:
# independent chains of dependent multiply-adds on a full grid, no memory
# traffic).  Beside it, the rate the ncu counters suggest: a warp-wide
# IMAD.WIDE.U32 keeps the FMA-heavy pipe of its SM sub-partition busy for 4
# cycles (fmaheavy busy cycles against the per-opcode counts), i.e. 8 wide
# multiplies per clock per sub-partition, 4 sub-partitions per SM.
WIDE_MUL_PER_SPIN = 5
WIDE_MUL_PER_CLK_PER_SMSP = 8
SMSP_PER_SM = 4


def mulwide_rate(ising, torch, stream, form, iters=16384, reps=10):
    """One form of the wide-multiply probe, timed with CUDA events on its
    stream after warm-up launches: multiplies per second (median launch)."""
    sink = torch.zeros(1, dtype=torch.int64, device=stream.device)
    torch.cuda.synchronize()
    for _ in range(3):
        n = ising.ising_mulwide_probe(form, iters, sink, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(reps):
            ising.ising_mulwide_probe(form, iters, sink, stream)
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    times = [ev[k].elapsed_time(ev[k + 1]) for k in range(reps)]
    med = statistics.median(times)
    return {"t_mul_per_s": round(n / (med * 1e-3) / 1e12, 3), "t_mul_per_s_best": round(n / (min(times) * 1e-3) / 1e12, 3),
            "ms_median": round(med, 4), "multiplies_per_launch": n, "launches": reps}


def mulwide_peak(ising, torch, stream):
    """Measured peak of the 32 x 32 -> 64-bit multiply in the form a Philox
    round issues it (form 0), with the register-addend form beside it."""
    philox_form = mulwide_rate(ising, torch, stream, 0)
    addend_form = mulwide_rate(ising, torch, stream, 1)
    return dict(philox_form, kernel="mulwide_probe_kernel<0>: 16 chains per thread of x = hi ^ lo of "
                "mul.wide.u32(x, immediate), full grid", addend_form=addend_form)


def source_digest() -> str:
    """Hash of the sweep kernel's sources, to tie an ncu traffic figure to the
    exact kernel it was measured on."""
    import hashlib

    h = hashlib.sha256()
    for f in ("msc4.cu", "sweep_core.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1906_06297_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(L: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None), scaled by the spins per launch."""
    try:
        with open(os.path.join(ROOT, "profiles", "msc4_sweep_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None, None
    if rec.get("source_digest") != source_digest():
        return None, "stale"
    per_spin = rec["dram_bytes_per_launch"] / (rec["L"] * rec["L"] / 2)
    return round(per_spin * L * L / 2), f"ncu capture at L={rec['L']}, scaled by spins per launch"


def sweep_roofline(torch, device, L, plane_bytes, launch_ms, mul_peak=None):
    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    clk_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    derived_tmul = sms * SMSP_PER_SM * WIDE_MUL_PER_CLK_PER_SMSP * clk_hz / 1e12
    peak_tmul = mul_peak["t_mul_per_s"] if mul_peak else derived_tmul
    spins = L * L / 2
    achieved_tmul = WIDE_MUL_PER_SPIN * spins / (launch_ms * 1e-3) / 1e12
    alg_bytes = 3 * plane_bytes  # read + write the target plane, read the source plane
    hbm_gbs = alg_bytes / (launch_ms * 1e-3) / 1e9
    traffic, traffic_src = profiled_traffic(L)
    return {
        "bound": "alu", "achieved": round(achieved_tmul, 3), "peak": round(peak_tmul, 3),
        "unit": "T wide-mul/s", "frac": round(achieved_tmul / peak_tmul, 4), "traffic": traffic,
        "traffic_source": traffic_src,
        "peak_source": ("measured: wide-multiply probe on this GPU in this run (median of "
                        f"{mul_peak['launches']} launches)" if mul_peak else "derived (probe not run)"),
        "peak_probe": mul_peak,
        "peak_derived": {"t_mul_per_s": round(derived_tmul, 3),
                         "derivation": f"{sms} SMs x {SMSP_PER_SM} sub-partitions x {WIDE_MUL_PER_CLK_PER_SMSP} "
                                       f"IMAD.WIDE/clk x {clk_hz / 1e6:.0f} MHz"},
        "work_per_spin": f"{WIDE_MUL_PER_SPIN} wide multiplies per spin update (Philox4x32-10 per 4 draws; "
                         "every block computed, no skip of blocks whose 4 sites all have a <= 2)",
        "peak_flips_per_ns": round(peak_tmul * 1e12 / WIDE_MUL_PER_SPIN / 1e9, 1),
        "alg_bytes_per_launch": alg_bytes,
        "hbm": {"achieved": round(hbm_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(hbm_gbs / peaks["hbm_gbs"], 4), "peak_source": peak_kind},
    }


def time_sweeps(ising, torch, lat, beta, seed, steps, warmup, trace, stream, per_kernel=True):
    """Warm up, then time `steps` sweeps on `stream`.  Each step is two public
    calls (black half-sweep; white half-sweep with the fused trace row), with
    CUDA events around every launch.  Returns (total_ms, black_ms[], white_ms[])."""
    for k in range(warmup):
        ising.ising_half_sweep(lat, beta, 0, seed, k, None, stream)
        ising.ising_half_sweep(lat, beta, 1, seed, k, trace[k % trace.shape[0]], stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps + 1)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            t = warmup + k
            ising.ising_half_sweep(lat, beta, 0, seed, t, None, stream)
            ev[2 * k + 1].record(stream)
            ising.ising_half_sweep(lat, beta, 1, seed, t, trace[k], stream)
            ev[2 * k + 2].record(stream)
    torch.cuda.synchronize()
    black = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)]
    white = [ev[2 * k + 1].elapsed_time(ev[2 * k + 2]) for k in range(steps)]
    total = ev[0].elapsed_time(ev[2 * steps])
    return total, black, white


def sweep_config(args, world):
    """The `config` of the single-lattice line (one lattice per rank)."""
    L, plane_bytes = args.L, args.L * args.L // 4
    return {"workload": f"msc4 L={L} {args.init} start seed {args.seed}+rank beta={args.beta}, 1 sweep per step",
            "L": L, "layout": "msc4", "beta": args.beta, "spins": L * L, "plane_bytes": plane_bytes,
            "l2": f"inputs larger than L2 (two planes of {plane_bytes / 1e9:.2f} GB each), no flush",
            "parallelism": f"replicas{world}"}


def slab_config(args, world, seed):
    """The `config` of the slab line (one lattice cut into horizontal slabs)."""
    return {"workload": f"msc4 L={args.L} random start seed {seed} beta={args.beta} as "
                        f"{args.slabs if world == 1 else world} horizontal slabs with halo rows",
            "L": args.L, "layout": "msc4", "beta": args.beta, "parallelism": f"slabs{world}",
            "l2": "inputs larger than L2, no flush"}


def run_ours(args, world, rank, local):
    import torch

    import paper_1906_06297_gb300 as ising

    ising.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)

    L, beta = args.L, args.beta
    seed = replica_seed(args.seed, rank)
    n_sites = L * L
    stream = torch.cuda.Stream(device=device)
    lat = ising.Lattice(L, "msc4", device=device)
    mode = ising.ISING_INIT_RANDOM if args.init == "random" else ising.ISING_INIT_UP
    ising.ising_init_lattice(lat, mode, seed, stream)
    trace = torch.zeros((max(args.steps, args.warmup, 1), 2), dtype=torch.int64, device=device)
    torch.cuda.synchronize()

    barrier(world)
    with ClockSampler(local) as clk:
        total_ms, black, white = time_sweeps(ising, torch, lat, beta, seed, args.steps, args.warmup, trace, stream)
    clocks = clk.summary()
    barrier(world)
    max_ms = max_over_ranks(total_ms, world, device)
    value = world * n_sites * args.steps / (max_ms * 1e6)

    _, plane_bytes = ising.ising_lattice_bytes(L, ising.ISING_MSC4)
    launch_ms = statistics.mean(black + white)
    mul_peak = mulwide_peak(ising, torch, stream)
    roofline = sweep_roofline(torch, device, L, plane_bytes, launch_ms, mul_peak)
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "impl": "ours",
        "config": sweep_config(args, world),
        "gpu_launches": 2 * args.steps,
        "kernel_ms": {"black_mean": round(statistics.mean(black), 4), "white_mean": round(statistics.mean(white), 4),
                      "min": round(min(black + white), 4)},
        "roofline": roofline,
        "clocks": clocks,
        "context": PAPER_CONTEXT,
    }

    if rank == 0 and not args.no_extras:
        # per-beta rates (config: beta in {0.30, 0.4406868, 0.60})
        # 200 sweeps each; GB/s counts the algorithmic 1.5 bytes per spin update
        per_beta, per_beta_gbs = {}, {}
        ptrace = torch.zeros((200, 2), dtype=torch.int64, device=device)
        torch.cuda.synchronize()  # the fill precedes the sweeps on `stream`
        for b in (0.30, BETA_C_CONFIG, 0.60):
            tot, _, _ = time_sweeps(ising, torch, lat, b, seed, 200, 2, ptrace, stream, per_kernel=False)
            per_beta[str(b)] = round(n_sites * 200 / (tot * 1e6), 2)
            per_beta_gbs[str(b)] = round(1.5 * per_beta[str(b)], 1)
        del ptrace
        result["per_beta"] = per_beta
        result["per_beta_hbm_gbs"] = per_beta_gbs
        result["scale_leg"] = run_scale_leg(ising, torch, args, device, stream)
        result["rng_probe"] = rng_probe(ising, torch, L, seed, stream)
        result["e2e"] = run_e2e(ising, torch, args, L, beta, seed, device, stream)
        spot = None if args.cpu_short else gpu_spot(ising, torch, lat, L, beta, seed, stream)
        result["cpu_baseline"] = cpu_baseline(args, spot)
        if not args.no_batch:
            result["pt_batch"] = run_pt_batch(ising, torch, args, device, stream)
        if not args.no_learned:
            result["learned"] = run_learned(ising, torch, args, device, stream)
        result["slab_leg"] = run_slab_leg(ising, torch, args, device, stream, value / world)
        if not args.no_binder:
            result["binder"] = run_binder_leg(args, device, stream)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return result


def run_scale_leg(ising, torch, args, device, stream, L=262144, n=50):
    """The 262144^2 lattice (6.9e10 spins, two 17.2 GB planes) from a cold
    (all +1) start at beta = 0.4406868: 50 sweeps in one public call, timed
    with CUDA events, and the per-sweep energy and magnetisation per site
    beside the critical energy of Onsager's solution, -sqrt(2)."""
    import math

    lat = ising.Lattice(L, "msc4", device=device)
    ising.ising_init_lattice(lat, ising.ISING_INIT_UP, args.seed, stream)
    trace = torch.zeros((n, 2), dtype=torch.int64, device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        ising.ising_sweep(lat, BETA_C_CONFIG, n, args.seed, 0, trace, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h = trace.cpu().numpy()
    e = [-int(x) / (L * L) for x in h[:, 1]]
    m = [int(x) / (L * L) for x in h[:, 0]]
    del lat, trace
    torch.cuda.empty_cache()
    pick = [0, 1, 2, 4, 9, 19, 29, 39, 49]
    return {"workload": f"msc4 L={L} cold start, beta={BETA_C_CONFIG}, {n} sweeps in one ising_sweep call",
            "spins": L * L, "plane_bytes": L * L // 4, "ms": round(ms, 2),
            "flips_per_ns": round(L * L * n / (ms * 1e6), 2),
            "e_per_site": {str(i + 1): round(e[i], 6) for i in pick},
            "m_per_site": {str(i + 1): round(m[i], 6) for i in pick},
            "onsager_e_critical": round(-math.sqrt(2.0), 6),
            "note": "from the ordered start (e = -2, m = 1) the lattice relaxes towards the critical energy; "
                    "50 sweeps are far from equilibrium at this size (tau grows as L^2.17)"}


def time_slab_sweeps(ising, torch, slabs, beta, seed, steps, warmup, trace, stream):
    """K slabs of one lattice on this GPU (halo copies + per-slab half-sweeps,
    one public call per batch of sweeps): warm-up, then `steps` sweeps timed
    with CUDA events on `stream`.  Returns total ms."""
    ising.ising_slab_sweep(slabs, beta, warmup, seed, 0, trace[:max(warmup, 1)], stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        ising.ising_slab_sweep(slabs, beta, steps, seed, warmup, trace[:steps], stream)
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_slab_leg(ising, torch, args, device, stream, whole_flips_per_ns):
    """The lattice of the headline workload held as K horizontal slabs with
    halo rows on this GPU (Sec. 4 layout): flips/ns and the cost of the halo
    copies relative to the whole-lattice sweep."""
    L, k, steps = args.L, args.slabs, 20
    seed = replica_seed(args.seed, 0)
    slabs = []
    for row0, rows in ising.slab_partition(L, k):
        sl = ising.Slab(L, row0, rows, device=device)
        ising.ising_slab_init(sl, ising.ISING_INIT_RANDOM, seed, stream)
        slabs.append(sl)
    trace = torch.zeros((steps, 2), dtype=torch.int64, device=device)
    torch.cuda.synchronize()  # the fill precedes the sweeps on `stream`
    ms = time_slab_sweeps(ising, torch, slabs, args.beta, seed, steps, 3, trace, stream)
    rate = L * L * steps / (ms * 1e6)
    del slabs
    torch.cuda.empty_cache()
    return {"slabs": k, "L": L, "sweeps": steps, "flips_per_ns": round(rate, 2),
            "vs_whole_lattice": round(rate / whole_flips_per_ns, 4),
            "gpu_launches_per_sweep": 2 * (k + 1)}


def run_binder_leg(args, device, stream):
    """Binder cumulant crossing (Sec. 5.3, Fig. 6) of 64^2, 128^2 and 256^2
    lattices from the batched sampler with replica exchange: 8 ladders of 16
    betas in [0.42, 0.46] per size, all sizes in one batch."""
    import torch

    from paper_1906_06297_gb300 import binder

    sizes, ladders, S = (64, 128, 256), 8, 16
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = binder.binder_study(sizes=sizes, ladders=ladders, ladder_size=S, beta_lo=0.42, beta_hi=0.46,
                              sweeps=args.binder_sweeps, thermalize=args.binder_sweeps // 10, record_every=2,
                              chunks=10, seed=args.seed, device=device, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    spins = ladders * S * sum(x * x for x in sizes)
    total_sweeps = res["sweeps"] + res["thermalize"]
    return {"workload": f"sizes {list(sizes)}, {ladders} ladders x {S} betas in [0.42, 0.46] per size, "
                        f"exchange every 2 sweeps, {res['thermalize']} + {res['sweeps']} sweeps",
            "beta_c": round(binder.BETA_C, 7),
            "crossings": {k: [round(x, 5) for x in v] for k, v in res["crossings"].items()},
            "beta_nearest_c": round(res["beta_nearest_c"], 5),
            "U_at_beta_nearest_c": {k: round(v, 4) for k, v in res["U_at_beta_nearest_c"].items()},
            "U_err_max": {k: round(max(v), 4) for k, v in res["U_err"].items()},
            "ms": round(ms, 1), "flips_per_ns": round(spins * total_sweeps / (ms * 1e6), 1)}


def run_slabs(args, world, rank, local):
    """One L x L lattice cut into horizontal slabs (Sec. 4).  One process:
    args.slabs slabs on this GPU, halos by the library's copy kernel.  Several
    ranks: one slab per rank, halo rows exchanged point to point (NCCL) before
    each half-sweep, the trace all-reduced once at the end.  Strong scaling:
    the lattice is the same for every N."""
    import torch

    import paper_1906_06297_gb300 as ising

    ising.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    L, beta, seed = args.L, args.beta, args.seed
    stream = torch.cuda.Stream(device=device)
    n = max(args.steps, 1)
    trace = torch.zeros((n, 2), dtype=torch.int64, device=device)
    with torch.cuda.stream(stream):
        if world == 1:
            slabs = []
            for row0, rows in ising.slab_partition(L, args.slabs):
                sl = ising.Slab(L, row0, rows, device=device)
                ising.ising_slab_init(sl, ising.ISING_INIT_RANDOM, seed)
                slabs.append(sl)
            def step(count, off):
                ising.ising_slab_sweep(slabs, beta, count, seed, off, trace[:count])
            launches = 2 * (args.slabs + 1)
        else:
            row0, rows = ising.slab_partition(L, world)[rank]
            sl = ising.Slab(L, row0, rows, device=device)
            ising.ising_slab_init(sl, ising.ISING_INIT_RANDOM, seed)
            def step(count, off):
                ising.slab_sweep(sl, beta, count, seed, off, trace[:count])
            launches = 4
        step(max(args.warmup, 1), 0)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        e0.record(stream)
        step(args.steps, args.warmup)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    max_ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    value = L * L * args.steps / (max_ms * 1e6)
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "ours",
        "config": slab_config(args, world, seed),
        "gpu_launches": launches * args.steps,
        "clocks": clk.summary(),
    }
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return res


def rng_probe(ising, torch, L, seed, stream):
    """The generator alone: one Philox4x32-10 block per 4 sites of a
    half-sweep, each word compared with the a = 3 threshold and counted."""
    n_blocks = L * L // 8
    T3 = ising.ising_thresholds(BETA_C_CONFIG)[3]
    cnt = torch.zeros(1, dtype=torch.int64, device=stream.device)
    torch.cuda.synchronize()  # the fill precedes the counting on `stream`
    for _ in range(3):
        ising.ising_rng_probe(n_blocks, seed, 0, 0, T3, cnt, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    with torch.cuda.stream(stream):
        e0.record(stream)
        for k in range(reps):
            ising.ising_rng_probe(n_blocks, seed, k, 0, T3, cnt, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    rate = 4 * n_blocks / (ms * 1e6)
    return {"half_sweep_sites_per_ns": round(rate, 1), "ms": round(ms, 4), "flips_per_ns_ceiling": round(rate, 1),
            "kernel": "rng_probe_kernel: 8 Philox blocks per thread step sharing counter words 1..3, 32-bit "
                      "indices, full grid; one compare per draw",
            "t_mul_per_s_algorithmic": round(rate * WIDE_MUL_PER_SPIN / 1e3, 3)}


def run_e2e(ising, torch, args, L, beta, seed, device, stream):
    """Through the host-buffer entry points: every step copies the lattice in
    from pinned host memory, sweeps once, and copies lattice and trace back.
    The headline uses the bit-packed host format (ising_sweep_host_bits: one
    bit per spin on the link, converted to and from MSC4 on the device); the
    same sweep with MSC4 host planes (ising_sweep_host, four bits per spin on
    the link) is reported beside it."""
    steps = max(1, args.e2e_steps)
    dev = ising.Lattice(L, "msc4", device=device)
    ising.ising_init_lattice(dev, ising.ISING_INIT_RANDOM, seed, stream)
    nb = ising.ising_bits_bytes(L)
    stage = torch.empty(2 * nb, dtype=torch.uint8, device=device)
    ising.ising_msc4_to_bits(dev, stage[:nb], stage[nb:], stream)
    torch.cuda.synchronize()
    bb = stage[:nb].cpu().pin_memory()
    bw = stage[nb:].cpu().pin_memory()
    hb = dev.black.cpu().pin_memory()
    hw = dev.white.cpu().pin_memory()
    tr_dev = torch.zeros((1, 2), dtype=torch.int64, device=device)
    tr_host = torch.zeros((1, 2), dtype=torch.int64).pin_memory()

    def bits_step(k):
        ising.ising_sweep_host_bits(dev, bb, bw, stage, beta, 1, seed, k, tr_dev, tr_host.data_ptr(), stream)

    def msc4_step(k):
        ising.ising_sweep_host(dev, hb.data_ptr(), hw.data_ptr(), beta, 1, seed, k, tr_dev, tr_host.data_ptr(),
                               stream)

    def timed(step):
        for k in range(3):  # warm-up calls (sweep offsets 0..2), not timed
            step(k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for k in range(steps):
                step(3 + k)
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ms = timed(bits_step)
    ms4 = timed(msc4_step)
    plane = dev.row_bytes * L
    return {"value": round(L * L * steps / (ms * 1e6), 3), "unit": UNIT, "h2d_bytes_per_step": 2 * nb,
            "d2h_bytes_per_step": 2 * nb + 16, "steps": steps, "ms_per_step": round(ms / steps, 3),
            "host_format": "bit-packed planes, 1 bit per spin (ising_sweep_host_bits)",
            "msc4_host": {"value": round(L * L * steps / (ms4 * 1e6), 3), "unit": UNIT,
                          "h2d_bytes_per_step": 2 * plane, "d2h_bytes_per_step": 2 * plane + 16,
                          "ms_per_step": round(ms4 / steps, 3),
                          "host_format": "MSC4 planes, 4 bits per spin (ising_sweep_host)"}}


def run_pt_batch(ising, torch, args, device, stream):
    """The batched form: 4096 lattices (sides 32..1024, 8:8:4:2:1:1) in 64
    ladders of 64 temperatures in [0.30, 0.60], exchanges every 10 sweeps,
    all sweeps in one persistent launch replayed from a captured graph.
    Compared with looping the one-byte-per-spin single-lattice kernel over the
    same lattices, and, at the temperature nearest beta_c, effective samples
    per second of the side-32 ladders against the same lattices swept without
    exchanges."""
    import numpy as np

    from paper_1906_06297_gb300 import analysis, workloads

    L, S, beta = workloads.pt_batch()
    spins = int(sum(x * x for x in L))
    seed, every, warm = args.seed, 10, 20
    b = ising.Batch(L, S, beta, device=device)
    b.init(ising.ISING_INIT_RANDOM, seed, stream)
    threads, wpt = b.autotune(2, stream)
    args._pt_tuned = (threads, wpt)
    b.run(warm, seed, 0, every, True, None, True, stream)
    b.check(stream)
    sweeps = args.pt_sweeps
    n_ev = b.n_events(sweeps, warm, every)
    tr = torch.zeros((n_ev, len(L), 2), dtype=torch.int64, device=device)
    torch.cuda.synchronize()  # the fill precedes the run on `stream`
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.run(sweeps, seed, warm, every, True, tr, True, stream)
        e1.record(stream)
    b.check(stream)
    ms = e0.elapsed_time(e1)
    out = {"workload": f"{len(L)} lattices, sides {sorted(set(L))}, ladders of {S} betas in [0.30, 0.60], "
                       f"exchange every {every} sweeps, {sweeps} sweeps in one persistent launch (graph)",
           "spins": spins, "sweeps": sweeps, "ms": round(ms, 2), "flips_per_ns": round(spins * sweeps / (ms * 1e6), 1),
           "autotuned": {"threads": threads, "words_per_thread": wpt}, "gpu_launches": 1}
    del tr, b
    # looping the single-lattice one-byte-per-spin kernel over the same lattices
    lats = [ising.Lattice(x, "int8", device=device) for x in L]
    for i, lat in enumerate(lats):
        ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed + i, stream)
    loop_sweeps = 2
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for i, lat in enumerate(lats):
            ising.ising_sweep(lat, float(beta[i % S]), loop_sweeps, seed + i, 0, None, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1)
    out["loop_int8_per_lattice"] = {"flips_per_ns": round(spins * loop_sweeps / (loop_ms * 1e6), 2),
                                    "gpu_launches": 2 * loop_sweeps * len(L)}
    out["speedup_vs_loop"] = round(out["flips_per_ns"] / out["loop_int8_per_lattice"]["flips_per_ns"], 1)
    del lats
    out["matched_error"] = pt_matched_error(ising, torch, args, device, stream)
    return out


def pt_matched_error(ising, torch, args, device, stream):
    """Replica exchange against the plain sweep at matched observable error,
    per lattice side of the batch, at the ladder temperature nearest beta_c.

    Both runs sweep the whole 4096-lattice batch in the same persistent
    kernel, with and without exchanges: after `pt_ess_warm` sweeps, records
    every 10 sweeps for `pt_ess_sweeps` sweeps.  For each side L the series of
    |m| and e at slot k* (nearest beta_c) are taken per ladder: with exchanges
    the slot's trajectory across replicas, without them the lattice that stays
    at k*.  Cost of one record of one chain at beta*, from each run's measured
    rate R (flips/ns): plain, the chain's own 10 sweeps (a plain sweep can give
    the whole GPU to chains at beta*): 10 L^2 / R; with exchanges, its whole
    ladder's 10 sweeps and the exchanges: 10 S L^2 / R.  The time to a
    standard error of 1% of the mean (the same eps for both methods) then
    follows from each method's tau_int and variance (analysis.seconds_to_error)."""
    import numpy as np

    from paper_1906_06297_gb300 import analysis, workloads

    L, S, beta = workloads.pt_batch()
    spins = int(sum(x * x for x in L))
    every, seg = 10, 10000
    k = int(np.argmin(np.abs(beta - 0.5 * np.log(1 + np.sqrt(2)))))
    n_lad = len(L) // S
    side = np.array([L[l * S] for l in range(n_lad)])
    sweeps = max(seg, (args.pt_ess_sweeps // seg) * seg)
    runs = {}
    for name, swaps in (("exchange", True), ("plain", False)):
        b = ising.Batch(L, S, beta, device=device)
        b.init(ising.ISING_INIT_RANDOM, args.seed + 7, stream)
        if getattr(args, "_pt_tuned", None):
            b.config(*args._pt_tuned)
        else:
            b.autotune(2, stream)
        b.run(args.pt_ess_warm, args.seed + 7, 0, every, swaps, None, True, stream)
        b.check(stream)
        rows, ms = [], 0.0
        n_ev = b.n_events(seg, 0, every)
        tr = torch.zeros((n_ev, len(L), 2), dtype=torch.int64, device=device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for j in range(sweeps // seg):
            off = args.pt_ess_warm + j * seg
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                e0.record(stream)
                b.run(seg, args.seed + 7, off, every, swaps, tr, True, stream)
                e1.record(stream)
            b.check(stream)
            ms += e0.elapsed_time(e1)
            rows.append(tr[:, k::S, :].cpu().numpy())  # slot k* of every ladder
        runs[name] = {"h": np.concatenate(rows), "rate": spins * sweeps / (ms * 1e6), "ms": ms}
        del tr, b
    out = {"beta": round(float(beta[k]), 5), "sweeps": sweeps, "warm": args.pt_ess_warm, "record_every": every,
           "eps": "1% of the mean (same eps for both methods)",
           "rate_flips_per_ns": {n: round(r["rate"], 1) for n, r in runs.items()}, "sides": {}}
    for Lside in sorted(set(side.tolist())):
        lads = np.nonzero(side == Lside)[0]
        area = float(Lside * Lside)
        res = {"chains_at_beta": int(lads.size)}
        for obs, col, f in (("abs_m", 0, lambda v: np.abs(v) / area), ("e", 1, lambda v: -v / area)):
            series = {n: [f(r["h"][:, l, col].astype(np.float64)) for l in lads] for n, r in runs.items()}
            eps = 0.01 * abs(float(np.mean(np.concatenate(series["plain"]))))
            per = {}
            for n, r in runs.items():
                records = r["h"].shape[0] * lads.size
                per_record = every * area * (S if n == "exchange" else 1) / (r["rate"] * 1e9)
                st = analysis.seconds_to_error(series[n], records * per_record, eps)
                per[n] = {"seconds_to_error": round(st["seconds_to_error"], 6),
                          "tau_int_sweeps": round(st["tau_int"] * every, 1), "mean": round(st["mean"], 5),
                          "series_over_tau": round(st["series_over_tau"], 1), "reliable": st["reliable"]}
            per["plain_over_exchange"] = round(per["plain"]["seconds_to_error"] /
                                               max(per["exchange"]["seconds_to_error"], 1e-30), 4)
            res[obs] = per
        out["sides"][str(Lside)] = res
    return out


def run_pt_only(args, world, rank, local):
    """Only the batched leg (one timed persistent launch of --pt-sweeps sweeps;
    with --no-extras no loop or effective-sample runs): used for profiling."""
    import torch

    import paper_1906_06297_gb300 as ising
    from paper_1906_06297_gb300 import workloads

    ising.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=device)
    if args.no_extras:
        L, S, beta = workloads.pt_batch()
        b = ising.Batch(L, S, beta, device=device)
        b.init(ising.ISING_INIT_RANDOM, args.seed, stream)
        tuned = b.autotune(2, stream)
        b.run(10, args.seed, 0, 10, True, None, True, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            torch.cuda.nvtx.range_push("pt_timed")  # lets a profiler select the timed launch
            e0.record(stream)
            b.run(args.pt_sweeps, args.seed, 10, 10, True, None, True, stream)
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
        b.check(stream)
        ms = e0.elapsed_time(e1)
        spins = int(sum(x * x for x in L))
        pt = {"spins": spins, "sweeps": args.pt_sweeps, "ms": round(ms, 3),
              "flips_per_ns": round(spins * args.pt_sweeps / (ms * 1e6), 1),
              "autotuned": {"threads": tuned[0], "words_per_thread": tuned[1]}}
    else:
        pt = run_pt_batch(ising, torch, args, device, stream)
    return {"metric": METRIC, "value": pt["flips_per_ns"], "unit": UNIT, "n_gpus": world, "impl": "ours",
            "config": {"workload": "parallel-tempering batch (4096 lattices, 64 ladders x 64 betas)"},
            "pt_batch": pt}


def time_network(ising, torch, L, C, params, beta, seed, device, stream, reps=10, warmup=3):
    """CUDA-event times of one network evaluation of C chains of side L: the
    full forward (the state before a move) and the flipped-band forward (the
    proposed state), with the tensor-core FLOPs of the two 32 -> 32 layers."""
    import numpy as np

    mv = ising.BlockMove(L, C, beta, device=device)
    mv.batch.init(ising.ISING_INIT_RANDOM, seed, stream)
    mv.batch.run(20, seed, 0, 0, False, None, True, stream)
    nb = (L // 8) ** 2
    flips = torch.from_numpy(np.random.default_rng(seed).integers(0, nb, C).astype(np.int32)).to(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, fn in (("full_forward", lambda: ising.ising_net_forward(L, C, mv.black, mv.white, None, params, mv.lx,
                                                                      mv.work, False, stream)),
                     ("flipped_band_forward", lambda: ising.ising_net_forward_flipped(
                         L, C, mv.black, mv.white, flips, params, mv.lx, mv.lxp, mv.work, stream))):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms"] = round(e0.elapsed_time(e1) / reps, 4)
    ising.ising_net_check(stream)
    px = C * L * L
    conv_flops = 2 * 2 * (9 * 32) * 32 * px  # two 32 -> 32 layers, 2 flops per multiply-add
    # algorithmic HBM traffic of a full inference forward (layer 1 is formed inside the first
    # conv, so a1 never reaches HBM): a2 (bfloat16, rows of L + 2 pixels) written once and read
    # once, the row partials of z4 (9 FP32 values per row and 8-pixel block column) written and
    # read, the spins and the logits; the conv layers' operands are below the GB300 ridge
    # (~280 FLOP/B), so HBM is the roofline
    act = C * L * (L + 2) * 64
    alg_bytes = 2 * act + 2 * 9 * 4 * (px // 8) + px // 2 + C * (L // 8) ** 2 * 4
    peaks, source = measured_peaks()
    t = out["full_forward_ms"] * 1e-3
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    tensor_peak = float(peaks.get("bf16_tflops", 1900.0))
    out["conv_tflop_per_forward"] = round(conv_flops / 1e12, 4)
    out["alg_bytes_per_forward"] = alg_bytes
    out["roofline"] = {
        "bound": "hbm", "achieved": round(alg_bytes / t / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
        "frac": round(alg_bytes / t / 1e9 / hbm_peak, 4), "peak_source": source,
        "tensor": {"achieved": round(conv_flops / t / 1e12, 2), "peak": tensor_peak, "unit": "TFLOP/s",
                   "frac": round(conv_flops / t / 1e12 / tensor_peak, 4), "peak_source": f"bf16 burst, {source}"},
        "note": "whole inference forward (4 kernels at L a multiple of 128): algorithmic bytes and tensor-core FLOPs over the CUDA-event time"}
    del mv
    return out


def run_learned(ising, torch, args, device, stream):
    """The learned form at beta_c on 1024 chains of 128 x 128: train the
    proposal network on configurations from the plain sweep (10 sweeps apart),
    then compare, from the same starting states, cycles of (one sweep) with
    cycles of (one sweep + one uniform block move) and (one sweep + one network
    block move): integrated autocorrelation times per cycle of |m| and E, their
    effective samples per GPU second, and block acceptance rates."""
    import numpy as np

    from paper_1906_06297_gb300 import analysis

    L, beta, seed = 128, BETA_C_CONFIG, args.seed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tr = ising.train_block_proposer(L, beta, n_configs=args.learned_configs, batch=64, steps=args.learned_steps,
                                    lr=2e-3, seed=seed, log_every=max(1, args.learned_steps // 10), device=device,
                                    stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    C, cycles, warm = args.learned_chains, args.learned_cycles, 5000
    net = time_network(ising, torch, L, C, tr["params"], beta, seed, device, stream)
    variants, series = {}, {}
    for name in ("plain", "uniform", "learned"):
        mv = ising.BlockMove(L, C, beta, device=device)
        mv.batch.init(ising.ISING_INIT_RANDOM, seed, stream)
        mv.batch.run(warm, seed, 0, 0, False, None, True, stream)
        trace = torch.zeros((cycles, C, 2), dtype=torch.int64, device=device)
        # the move writes each cycle's acceptance flags straight into its row
        acc_rows = torch.zeros((cycles, C), dtype=torch.int32, device=device)
        params = tr["params"] if name == "learned" else None
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for k in range(cycles):
                t = warm + k
                mv.batch.run(1, seed, t, 1, False, trace[k], True, stream)
                if name != "plain":
                    mv.accepted = acc_rows[k]
                    mv.move(params, seed, t, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        h = trace.cpu().numpy()
        m = [np.abs(h[:, c, 0]) / (L * L) for c in range(C)]
        e = [-h[:, c, 1] / (L * L) for c in range(C)]
        em, ee = analysis.effective_samples(m), analysis.effective_samples(e)
        variants[name] = {"ms": round(ms, 2), "ms_per_cycle": round(ms / cycles, 4),
                          "tau_abs_m_cycles": round(em["tau_int"], 2), "tau_e_cycles": round(ee["tau_int"], 2),
                          "ess_per_s_abs_m": round(em["effective"] / (ms * 1e-3), 1),
                          "ess_per_s_e": round(ee["effective"] / (ms * 1e-3), 1),
                          "block_acceptance": (round(float(acc_rows.sum().item()) / (C * cycles), 5)
                                               if name != "plain" else None),
                          "mean_e": round(float(np.mean(np.concatenate(e))), 5)}
        series[name] = (m, e, ms * 1e-3)
        del mv, trace
    ising.ising_net_check(stream)
    # time to a standard error of 1% of the plain sweep's mean, the same eps
    # for every variant (matched observable error)
    for obs, j in (("abs_m", 0), ("e", 1)):
        eps = 0.01 * abs(float(np.mean(np.concatenate(series["plain"][j]))))
        for name in series:
            st = analysis.seconds_to_error(series[name][j], series[name][2], eps)
            variants[name][f"seconds_to_error_{obs}"] = round(st["seconds_to_error"], 6)
            variants[name][f"series_over_tau_{obs}"] = round(st["series_over_tau"], 1)
            variants[name][f"reliable_{obs}"] = st["reliable"]
        for name in ("uniform", "learned"):
            variants[name][f"time_ratio_vs_plain_{obs}"] = round(
                variants[name][f"seconds_to_error_{obs}"] / max(variants["plain"][f"seconds_to_error_{obs}"], 1e-30), 2)
    return {"workload": f"{C} chains of {L}x{L} at beta={beta}; network trained for {args.learned_steps} Adam steps "
                        f"(batch 64) on {args.learned_configs} plain-sweep configurations 10 sweeps apart; "
                        f"{cycles} measured cycles after {warm} sweeps",
            "train_ms": round(train_ms, 1), "train_loss_first_last": [round(tr["loss"][0], 4), round(tr["loss"][-1], 4)],
            "network": net, "variants": variants,
            "matched_error": "seconds_to_error_*: GPU seconds for a standard error of 1% of the plain sweep's mean "
                             "(the same eps for all three); time_ratio_vs_plain > 1 means slower than the plain sweep",
            "note": "reliable_*: each chain's series is at least 50 tau_int long"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def time_oracle(L, beta, sweeps, seed, threads):
    """One oracle run from the keyed random start: (flips/ns, seconds)."""
    import oracle

    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    t0 = time.perf_counter()
    oracle.run(s, beta, sweeps, seed, trace=True, nthreads=threads)
    dt = time.perf_counter() - t0
    return {"L": L, "sweeps": sweeps, "threads": threads, "flips_per_ns": round(L * L * sweeps / (dt * 1e9), 5),
            "s": round(dt, 2)}


def cpu_baseline(args, spot=None):
    """The oracle as it stands, on the host cores: bounded samples of the same
    workload (same beta and keyed random start).  The headline value is the
    16384^2 lattice on all cores; beside it the 256^2 parity workload (1000
    sweeps), one sweep of 16384^2 on one thread, and the at-scale spot check:
    two oracle sweeps of the full 65536^2 lattice compared with the GPU's
    trace and rows after the same two sweeps."""
    import oracle

    threads = oracle.max_threads()
    main = time_oracle(args.cpu_L, args.beta, args.cpu_sweeps, args.seed, threads)
    out = {"value": main["flips_per_ns"], "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"int8 L={args.cpu_L} random start seed {args.seed}, {args.cpu_sweeps} sweeps at "
                     f"beta={args.beta}, {threads} OpenMP threads ({main['s']:.1f} s)",
           "nproc": os.cpu_count(), "cpu_model": cpu_model(), "machine": os.uname().machine}
    if args.cpu_short:
        return out
    out["all_cores_L16384"] = main if args.cpu_L == 16384 else time_oracle(16384, args.beta, 20, args.seed, threads)
    out["one_thread_L16384"] = time_oracle(16384, args.beta, args.cpu_sweeps_1t, args.seed, 1)
    out["config1_L256"] = time_oracle(256, args.beta, 1000, args.seed, threads)
    if spot is not None:
        L, sweeps = spot["L"], spot["sweeps"]
        s = oracle.init(L, oracle.MODE_RANDOM, args.seed)
        t0 = time.perf_counter()
        tr = oracle.run(s, args.beta, sweeps, args.seed, trace=True, nthreads=threads)
        dt = time.perf_counter() - t0
        rows_equal = all(bool((oracle.row_from_planes_msc4(L, i, b, w) == s[i]).all())
                         for i, (b, w) in spot["rows"].items())
        out["spot_check_L65536"] = {
            "L": L, "sweeps": sweeps, "threads": threads, "s": round(dt, 2),
            "flips_per_ns": round(L * L * sweeps / (dt * 1e9), 5),
            "trace_equal": bool((tr == spot["trace"]).all()), "rows_checked": sorted(spot["rows"]),
            "rows_equal": rows_equal}
        del s
    return out


def gpu_spot(ising, torch, lat, L, beta, seed, stream, sweeps=2):
    """The GPU side of the at-scale spot check: the lattice re-initialised
    from the seed, `sweeps` sweeps with the trace, and a few rows copied back."""
    ising.ising_init_lattice(lat, ising.ISING_INIT_RANDOM, seed, stream)
    tr = torch.zeros((sweeps, 2), dtype=torch.int64, device=stream.device)
    ising.ising_sweep(lat, beta, sweeps, seed, 0, tr, stream)
    torch.cuda.synchronize()
    import numpy as np

    rows = {}
    for i in (0, 1, L // 2, L - 1):
        b = np.ascontiguousarray(lat.black[i, :lat.row_bytes].cpu().numpy()).view(np.uint64)
        w = np.ascontiguousarray(lat.white[i, :lat.row_bytes].cpu().numpy()).view(np.uint64)
        rows[i] = (b.copy(), w.copy())
    return {"L": L, "sweeps": sweeps, "trace": tr.cpu().numpy(), "rows": rows}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    import oracle

    if rank != 0:
        return None
    L = args.ref_L
    s = oracle.init(L, oracle.MODE_RANDOM, args.seed)
    threads = oracle.max_threads()
    for k in range(args.warmup):
        oracle.run(s, args.beta, 1, args.seed, off=k, trace=True, nthreads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.run(s, args.beta, 1, args.seed, off=args.warmup + k, trace=True, nthreads=threads)
    dt = time.perf_counter() - t0
    value = L * L * args.steps / (dt * 1e9)
    sample = (f"oracle (plain C, int8 full lattice) L={L} random start seed {args.seed}, beta={args.beta}, "
              f"1 sweep per step; bounded sample of the msc4 L={args.L} workload")
    return {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic", "impl": "reference",
        # the workload our arm runs at this world size; each step here is a bounded sample of it
        "config": sweep_config(args, world) if world == 1 else slab_config(args, world, args.seed),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main(argv=None):
    args = parse_args(argv)
    world, rank, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    elif args.workload == "pt":
        res = run_pt_only(args, world, rank, local)
    elif args.workload == "slabs" or (args.workload == "sweep" and world > 1):
        # several GPUs: one lattice cut into one horizontal slab per rank (Sec. 4)
        res = run_slabs(args, world, rank, local)
    elif args.workload == "probes":
        # the integer ceiling alone: wide-multiply probe (both forms) and the
        # Philox-only probe over the sites of one half-sweep of an L^2 lattice
        import torch

        import paper_1906_06297_gb300 as ising

        ising.build()
        torch.cuda.set_device(local)
        device = torch.device("cuda", local)
        stream = torch.cuda.Stream(device=device)
        with ClockSampler(local) as clk:
            mul = mulwide_peak(ising, torch, stream)
            rng = rng_probe(ising, torch, args.L, args.seed, stream)
        res = {"metric": "wide multiplies/s", "value": mul["t_mul_per_s"], "unit": "T/s", "impl": "ours",
               "higher_is_better": True,
               "config": {"workload": f"integer probes; Philox-only probe over {args.L}^2 / 2 sites"},
               "mulwide": mul, "rng_probe": rng,
               "rng_probe_frac_of_mul_peak": round(rng["t_mul_per_s_algorithmic"] / mul["t_mul_per_s"], 4),
               "clocks": clk.summary()}
    elif args.workload == "host":
        # the host-buffer legs alone: one sweep per step of the L^2 lattice
        # held in pinned host memory (bit-packed, and MSC4 beside it)
        import torch

        import paper_1906_06297_gb300 as ising

        ising.build()
        torch.cuda.set_device(local)
        device = torch.device("cuda", local)
        e2e = run_e2e(ising, torch, args, args.L, args.beta, args.seed, device, torch.cuda.Stream(device=device))
        res = {"metric": METRIC, "value": e2e["value"], "unit": UNIT, "impl": "ours",
               "config": {"workload": f"{args.L}x{args.L} MSC4 lattice in host memory, one sweep per step",
                          "beta": args.beta}, "e2e": e2e}
    elif args.workload == "binder":
        import torch

        import paper_1906_06297_gb300 as ising

        ising.build()
        torch.cuda.set_device(local)
        device = torch.device("cuda", local)
        bl = run_binder_leg(args, device, torch.cuda.Stream(device=device))
        res = {"metric": METRIC, "value": bl["flips_per_ns"], "unit": UNIT, "impl": "ours",
               "config": {"workload": bl["workload"]}, "binder": bl}
    elif args.workload == "network":
        # the network's forward passes alone (random weights): full and flipped band
        import numpy as np
        import torch

        import paper_1906_06297_gb300 as ising

        ising.build()
        torch.cuda.set_device(local)
        device = torch.device("cuda", local)
        rng = np.random.default_rng(args.seed)
        params = torch.from_numpy(rng.normal(0.0, 0.1, ising.ising_net_param_count()).astype(np.float32)).to(device)
        C = args.learned_chains
        net = time_network(ising, torch, 128, C, params, BETA_C_CONFIG, args.seed, device,
                           torch.cuda.Stream(device=device), reps=args.net_reps, warmup=min(3, args.warmup))
        res = {"metric": "network forward pixels/s", "value": round(C * 128 * 128 / net["full_forward_ms"] / 1e6, 3),
               "unit": "Gpixel/s", "impl": "ours", "higher_is_better": True,
               "config": {"workload": f"{C} chains of 128x128, random bfloat16 weights"}, "network": net}
    elif args.workload == "train":
        # the proposal network's training alone: --learned-steps Adam steps of batch 64 on
        # --learned-configs plain-sweep configurations of 128 x 128
        import torch

        import paper_1906_06297_gb300 as ising

        ising.build()
        torch.cuda.set_device(local)
        device = torch.device("cuda", local)
        stream = torch.cuda.Stream(device=device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tr = ising.train_block_proposer(128, BETA_C_CONFIG, n_configs=args.learned_configs, batch=64,
                                        steps=args.learned_steps, lr=2e-3, seed=args.seed,
                                        log_every=max(1, args.learned_steps // 10), device=device, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res = {"metric": "proposal-network training steps/s", "value": round(args.learned_steps / (ms * 1e-3), 2),
               "unit": "steps/s", "impl": "ours", "higher_is_better": True,
               "config": {"workload": f"{args.learned_steps} Adam steps, batch 64 chains of 128x128, "
                                      f"{args.learned_configs} configurations"},
               "train_ms": round(ms, 1), "loss_first_last": [round(tr["loss"][0], 4), round(tr["loss"][-1], 4)]}
    elif args.workload == "learned":
        import torch

        import paper_1906_06297_gb300 as ising

        ising.build()
        torch.cuda.set_device(local)
        device = torch.device("cuda", local)
        lr = run_learned(ising, torch, args, device, torch.cuda.Stream(device=device))
        res = {"metric": METRIC, "value": lr["variants"]["learned"]["ess_per_s_e"], "unit": "effective samples/s",
               "impl": "ours", "config": {"workload": lr["workload"]}, "learned": lr}
    else:
        res = run_ours(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
