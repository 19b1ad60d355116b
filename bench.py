"""Benchmark: point-halo grad+Hessian evaluations per second on the 2048^2,
1000-potential deflection + Hessian map (LENS_MIXED), plus the batched chi2
and FP64 comparison legs.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torch.distributed.run): every rank evaluates its own map of the
same size -- independent problems, no data-path collective ("weak" scaling);
value = all ranks' point-halo pairs / the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "point-halo grad+Hessian evals/s"
UNIT = "pair/s"
MAP_N, N_HALO = 2048, 1000
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2, written between timed steps

# FP32-pipe lane operations (FFMA + FADD + FMUL, each paired FFMA2 / FADD2 /
# FMUL2 counting two) and MUFU (XU pipe) instructions per point-halo pair of
# the lens arithmetic of the LENS_MIXED Hessian map kernel, from ncu on the
# 2048^2 x 1000 workload (the counter group of the map kernel's summary
# under profiles/: 65.0 lane operations per pair, of which 2.0 are the
# magnitude sum that decides the double-float repair); the compensated-fold
# overhead (~1 op per pair) is included.
FP32_OPS_PER_PAIR = 63.0
MUFU_OPS_PER_PAIR = 6.03
# every FP32 lane operation of the map call per pair: the kernel's 65.0 and
# the double-float repair kernel's 1.27 (same capture)
CALL_FP32_OPS_PER_PAIR = 66.3
# the same count for the potential-map kernel (ncu, same workload)
POT_FP32_OPS_PER_PAIR = 48.9
# DRAM bytes (read + write) of one launch of that kernel on that workload,
# from the same ncu capture; the 100.7 MB of output are partly still in L2
# when the kernel ends
MAP_TRAFFIC_BYTES = 352000 + 39027968
SMS, FP32_LANES, MUFU_LANES = 152, 128, 16
# FP64 FMA lanes per SM and clock (measured on this GPU: 1/64 of the FP32 rate)
FP64_LANES = 2
# Thread operations per model of the batched chi2 legs (ncu instruction
# counters on the 1000-potential model, 372 images; summary under profiles/):
# FP32 = FFMA + FADD + FMUL, FP64 = DFMA + DADD + DMUL, MUFU = XU pipe.
# Source-plane chi2, 4096 sets (k_chi2_source):
CHI2_SRC_OPS = {"fp32": 1.276e6, "fp64": 1.658e4, "mufu": 1.168e4}
# Image-plane chi2, 1024^2 grid, 256 sets (k_img_sources + search + the
# refinement's point-list kernels + dedup + polish + chi2, per model):
CHI2_IMG_OPS = {"fp32": 1.014e9, "fp64": 1.20e6, "mufu": 5.67e7}


def hbm_peak_gbs():
    """The measured copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json
    beside this file), else the fallback figure; and which it is."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "measured"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the chi2 / FP64 comparison legs")
    ap.add_argument("--profile-leg", default=None,
                    choices=["map", "potential", "chi2_source", "chi2_image", "mcmc", "scaled"],
                    help="run only this workload `--steps` times (for ncu launch lists); prints nothing")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9 for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def slowest_rank(pg, device, *times):
    """Max over ranks of each per-rank time (whole-job throughput is bounded
    by the slowest rank); identity without a process group."""
    if pg is None:
        return times
    import torch
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return tuple(float(x) for x in t.tolist())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_map_sample(m, g, seconds):
    """Time the oracle's Hessian map on row bands of the grid until ~seconds of
    CPU work; returns (pairs/s, rows evaluated, threads)."""
    import oracle
    nx = g["nx"]
    dy = (g["ymax"] - g["ymin"]) / (g["ny"] - 1)
    rows, pairs, t_used = 0, 0, 0.0
    band = 4
    while t_used < seconds and rows < g["ny"]:
        gb = dict(g, ymin=g["ymin"] + rows * dy, ymax=g["ymin"] + (rows + band - 1) * dy, ny=band)
        t0 = time.perf_counter()
        oracle.maps(m, gb, 1.0, 6)
        t_used += time.perf_counter() - t0
        rows += band
        pairs += band * nx * len(m)
        band = min(band * 2, 64)
    return pairs / t_used, rows, oracle.num_threads()


def leg_roofline(ops, models_per_s, f_hz):
    """Achieved operation rates of a chi2 leg from its per-model counts,
    against the FP32, FP64 and MUFU pipes' peaks at clock f_hz."""
    out = {"bound": "alu", "unit": "Top/s", "ops_per_model": ops, "source": "ncu instruction counters"}
    for pipe, lanes in (("fp32", FP32_LANES), ("fp64", FP64_LANES), ("mufu", MUFU_LANES)):
        ach = ops[pipe] * models_per_s / 1e12
        peak = SMS * lanes * f_hz / 1e12
        out[pipe] = {"achieved": ach, "peak": peak, "frac": ach / peak}
    return out


def interp_range_fraction(m, g, sub=64):
    """Fraction of (grid node, FP32 dPIE) pairs whose core-minus-cut
    arguments leave the range of the map kernel's interpolants
    (max(w_x^2, w_y^2) >= 0.16, where the kernel calls the library atan /
    log1p), on a sub x sub lattice of grid nodes, in FP64.  w_x and w_y are
    the tangents of the differences of the core and cut terms' atan / atanh
    arguments; potentials with b0 >= 5" (the FP64 path) are left out.  A
    workload diagnostic only."""
    t = np.asarray(m, dtype=np.float64)
    t = t[(t[:, 0] == 0) & (t[:, 7] < 5.0)]
    X, Y = np.meshgrid(np.linspace(g["xmin"], g["xmax"], sub), np.linspace(g["ymin"], g["ymax"], sub))
    X, Y = X.ravel()[:, None], Y.ravel()[:, None]
    x0, y0, th, e, rc, rt = (t[:, k][None, :] for k in (1, 2, 3, 4, 5, 6))
    c, s = np.cos(th), np.sin(th)
    x = c * (X - x0) + s * (Y - y0)
    y = -s * (X - x0) + c * (Y - y0)
    q = (1 - e) / (1 + e)
    u = 2 * np.sqrt(e) / (1 + e)
    sc, st = rc * (1 + e), rt * (1 + e)
    pc = np.sqrt(q * q * (sc * sc + x * x) + y * y)
    pt = np.sqrt(q * q * (st * st + x * x) + y * y)
    ac, at = u * x / (pc + sc), u * x / (pt + st)
    bc, bt = u * y / (pc + q * q * sc), u * y / (pt + q * q * st)
    wx = (ac - at) / (1 + ac * at)
    wy = (bc - bt) / (1 - bc * bt)
    return float(np.mean(np.maximum(wx * wx, wy * wy) >= 0.16))


def map_errors(res, m, g, dls=1.0, n=4000, seed=7):
    """Max error of a LENS_MIXED Hessian map (planes ax, ay, kappa, gamma1,
    gamma2, mu; a torch tensor on the device) against the oracle, on n random
    grid nodes, the corners, and a 48 x 48 block around the map's smallest
    deflection (where alpha's tolerance turns absolute).  Run outside any
    timed region."""
    import oracle
    import torch
    ny, nx = g["ny"], g["nx"]
    rng = np.random.default_rng(seed)
    ii, jj = rng.integers(0, nx, n), rng.integers(0, ny, n)
    ii[:4], jj[:4] = [0, nx - 1, 0, nx - 1], [0, 0, ny - 1, ny - 1]
    j0, i0 = divmod(int(torch.argmin(torch.hypot(res[0], res[1]))), nx)
    j0, i0 = min(max(j0 - 24, 0), max(ny - 48, 0)), min(max(i0 - 24, 0), max(nx - 48, 0))
    jb, ib = np.meshgrid(np.arange(j0, min(j0 + 48, ny)), np.arange(i0, min(i0 + 48, nx)), indexing="ij")
    ii, jj = np.concatenate([ii, ib.ravel()]), np.concatenate([jj, jb.ravel()])
    dx, dy = (g["xmax"] - g["xmin"]) / (nx - 1), (g["ymax"] - g["ymin"]) / (ny - 1)
    ev = oracle.model_eval(m, g["xmin"] + ii * dx, g["ymin"] + jj * dy, dls)
    rk, rg1, rg2 = 0.5 * (ev[:, 2] + ev[:, 3]), 0.5 * (ev[:, 2] - ev[:, 3]), ev[:, 4]
    rdet = (1 - rk) ** 2 - rg1 ** 2 - rg2 ** 2
    got = res[:, torch.from_numpy(jj).to(res.device), torch.from_numpy(ii).to(res.device)].double().cpu().numpy()
    ra = np.hypot(ev[:, 0], ev[:, 1])
    peak = ra.max()
    ea = np.hypot(got[0] - ev[:, 0], got[1] - ev[:, 1])
    tol_a = 1e-6 * np.maximum(ra, 1e-3 * peak)
    det = 1.0 / got[5]
    big = np.abs(rdet) >= 1e-2
    worst = int(np.argmax(ea / tol_a))
    out = {"nodes": int(len(ii)), "sample": f"{n} random nodes + corners + 48x48 block around min |alpha|",
           "alpha_abs_arcsec": float(ea.max()), "alpha_rel_max": float(np.max(ea / np.maximum(ra, 1e-3 * peak))),
           "alpha_worst_node": {"i": int(ii[worst]), "j": int(jj[worst]), "alpha_ref": float(ra[worst]),
                                "err": float(ea[worst])},
           "kappa": float(np.max(np.abs(got[2] - rk) / np.maximum(np.abs(rk), 1))),
           "gamma1": float(np.max(np.abs(got[3] - rg1) / np.maximum(np.abs(rg1), 1))),
           "gamma2": float(np.max(np.abs(got[4] - rg2) / np.maximum(np.abs(rg2), 1))),
           "det_abs": float(np.max(np.abs(det - rdet))),
           "mu_rel_where_det_ge_1e-2": float(np.max(np.abs(got[5] * rdet - 1.0)[big])) if big.any() else None,
           "tolerance": {"alpha": "1e-6 max(|a|, 1e-3 peak)", "kappa_gamma": "1e-5 max(|x|,1)",
                         "det_abs": "3e-5 + 2^-24 |det| (mu stored as FP32)", "chi2_rel": 1e-8},
           "within_tolerance": bool(np.all(ea <= tol_a)
                                    and np.all(np.abs(got[2] - rk) <= 1e-5 * np.maximum(np.abs(rk), 1))
                                    and np.all(np.abs(got[3] - rg1) <= 1e-5 * np.maximum(np.abs(rg1), 1))
                                    and np.all(np.abs(got[4] - rg2) <= 1e-5 * np.maximum(np.abs(rg2), 1))
                                    and np.all(np.abs(det - rdet) <= 3e-5 + 2.0 ** -24 * np.abs(rdet)))}
    return out


def run_reference(args, rank):
    """The oracle as it stands, on the host cores: each step a bounded row
    band of the same 2048^2 x 1000 workload."""
    if rank != 0:
        return
    from paper_2004_06352_gb300 import inputs as I
    import oracle
    oracle.build()
    m, g = I.cfg2_model(), I.grid(MAP_N)
    per_step_s = 4.0
    for _ in range(args.warmup):
        oracle_map_sample(m, g, 0.5)
    rates, rows = [], 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, nr, thr = oracle_map_sample(m, g, per_step_s)
        rates.append(r)
        rows += nr
    wall = time.perf_counter() - t0
    value = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "hessian_map 2048x2048 grid x 1000 dPIE potentials (2 cluster + 998 members)",
                       "sample": f"{rows} grid rows of 2048 across the steps"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"{rows} rows x 2048 points x 1000 potentials, FP64 C, OpenMP"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.profile_leg:
        profile_leg(args)
        return
    import torch
    from paper_2004_06352_gb300 import build as B
    B.build()
    from paper_2004_06352_gb300 import api
    from paper_2004_06352_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    m, g = I.cfg2_model(seed=2 + rank), I.grid(MAP_N)
    pairs = MAP_N * MAP_N * N_HALO
    ctx = api.Context(local)
    mid = ctx.model_upload(m)
    out = torch.empty((6, MAP_N, MAP_N), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ctx.hessian_map(mid, g, 1.0, api.LENS_MIXED, out, stream)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.hessian_map(mid, g, 1.0, api.LENS_MIXED, out, stream)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    kms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(kms))

    # end to end through the public API: host halo table -> upload -> map
    # streamed band by band into pinned host memory (all six planes), every step
    host = torch.empty((6, MAP_N, MAP_N), dtype=torch.float32, pin_memory=True)
    e2e_ms = []
    h2d_bytes = 0
    for k in range(args.warmup + args.steps):
        barrier()
        t1 = time.perf_counter()
        mid2 = ctx.model_upload(m)
        ctx.hessian_map_host(mid2, g, 1.0, api.LENS_MIXED, host, stream)
        ctx.wait(stream)
        dt = time.perf_counter() - t1
        # what lens_model_upload copies: the halo table (64-byte records) and
        # one int32 slot per potential; the records are built on the device
        h2d_bytes = len(m) * (api.HALO_BYTES + 4)
        ctx.model_release(mid2)
        if k >= args.warmup:
            e2e_ms.append(dt * 1e3)
    e2e_t = float(np.mean(e2e_ms))
    ms, e2e_t = slowest_rank(pg, dev, ms, e2e_t)
    value = ws * pairs / (ms * 1e-3)

    extra = {}
    if rank == 0:
        # accuracy of the timed map (its last step's output) against the oracle
        try:
            extra["max_err"] = {"hessian_map": map_errors(out, m, g)}
        except Exception as e:  # the line still prints without it
            extra["max_err"] = {"hessian_map": {"error": str(e)}}
    if rank == 0 and not args.no_extra:
        extra.update(extra_legs(ctx, api, I, torch, dev, m, g, mid, stream, extra["max_err"], out))

    if rank != 0:
        ctx.close()
        return
    f_max = (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    roof = {"bound": "alu", "unit": "Top/s", "traffic": MAP_TRAFFIC_BYTES}
    if FP32_OPS_PER_PAIR:
        ach = FP32_OPS_PER_PAIR * pairs / (ms * 1e-3) / 1e12
        peak = SMS * FP32_LANES * f_max / 1e12
        roof.update({"achieved": ach, "peak": peak, "frac": ach / peak,
                     "ops_per_pair": FP32_OPS_PER_PAIR, "pipe": "fp32 (FFMA/FADD/FMUL lanes)"})
        # the FP32 pipe's use by the whole call (magnitude sum and repair too)
        roof["call_ops_per_pair"] = CALL_FP32_OPS_PER_PAIR
        roof["call_frac"] = CALL_FP32_OPS_PER_PAIR * pairs / (ms * 1e-3) / 1e12 / peak
        if MUFU_OPS_PER_PAIR:
            mach = MUFU_OPS_PER_PAIR * pairs / (ms * 1e-3) / 1e12
            roof["mufu"] = {"achieved": mach, "peak": SMS * MUFU_LANES * f_max / 1e12,
                            "frac": mach / (SMS * MUFU_LANES * f_max / 1e12)}
    else:
        roof.update({"achieved": None, "peak": SMS * FP32_LANES * f_max / 1e12, "frac": None})
    # the map's DRAM traffic against the measured copy bandwidth (the output
    # planes are written once; the kernel is nowhere near this bound)
    hbm_peak, hbm_src = hbm_peak_gbs()
    hbm_ach = MAP_TRAFFIC_BYTES / (ms * 1e-3) / 1e9
    roof["hbm"] = {"achieved_gbs": hbm_ach, "peak_gbs": hbm_peak, "frac": hbm_ach / hbm_peak, "peak_source": hbm_src}
    cpu = extra.pop("cpu_baseline", None)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "hessian_map 2048x2048 grid x 1000 dPIE potentials (2 cluster FP64 + 998 "
                                   "members FP32), LENS_MIXED, outputs alpha_x, alpha_y, kappa, gamma1, gamma2, mu",
                       "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{ws}"},
            "e2e": {"value": ws * pairs / (e2e_t * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": 6 * MAP_N * MAP_N * 4},
            # per timed step one map kernel and one repair kernel (the
            # repair launches whatever the length of its list)
            "gpu_launches": 2 * args.steps, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "wall_s_timed": wall, "extra": extra}
    print(json.dumps(line), flush=True)
    ctx.close()


def extra_legs(ctx, api, I, torch, dev, m, g, mid, stream, errs, out):
    """Secondary numbers: grad-only map, plain FP64 GPU map, batched chi2, and
    the oracle on the host cores (bounded sample); max errors of the chi2 and
    potential outputs against the oracle go into errs."""
    ex = {}

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    pairs = MAP_N * MAP_N * N_HALO
    # the same map without the double-float repair of the near-zero nodes
    ctx.set_repair_ratio(0.0)
    t = timed(lambda: ctx.hessian_map(mid, g, 1.0, api.LENS_MIXED, out, stream), 5)
    ctx.set_repair_ratio(api.LENS_REPAIR_RATIO_DEFAULT)
    ex["hessian_map_no_repair"] = {"ms": t, "pair_per_s": pairs / (t * 1e-3),
                                   "workload": "as the headline map, repair ratio 0 (FP32 terms everywhere)"}
    ctx.hessian_map(mid, g, 1.0, api.LENS_MIXED, out, stream)
    out2 = torch.empty((2, MAP_N, MAP_N), dtype=torch.float32, device=dev)
    t = timed(lambda: ctx.grad_map(mid, g, 1.0, api.LENS_MIXED, out2, stream), 5)
    ex["grad_map_mixed"] = {"ms": t, "pair_per_s": pairs / (t * 1e-3)}
    del out2
    # the paper's own map benchmark shape (Sec. 5: a 5000^2 gradient map over
    # 150" x 150" of a 217-potential cluster model), with a synthetic model of
    # that size in place of its data: 2 cluster-scale halos + 215 members
    mp = I.cfg2_model(n_members=215)
    midp = ctx.model_upload(mp)
    gp = I.grid(5000, field=(-75.0, 75.0, -75.0, 75.0))
    out5 = torch.empty((2, 5000, 5000), dtype=torch.float32, device=dev)
    t = timed(lambda: ctx.grad_map(midp, gp, 1.0, api.LENS_MIXED, out5, stream), 5)
    pp = 5000 * 5000 * len(mp)
    ex["grad_map_paper_shape"] = {"ms": t, "pair_per_s": pp / (t * 1e-3),
                                  "workload": "gradient map 5000^2 over 150\" x 150\", 217 potentials "
                                              "(2 cluster + 215 members, synthetic), LENS_MIXED",
                                  "paper_p100_s": 0.93,
                                  "note": "the paper's 1-GPU time for its 217-potential model on this grid "
                                          "(P100, precision unstated; context, not a like-for-like comparison)"}
    del out5
    ctx.model_release(midp)
    # potential + time-delay (Fermat) surface about a source position
    outp = torch.empty((2, MAP_N, MAP_N), dtype=torch.float64, device=dev)
    t = timed(lambda: ctx.potential_map(mid, g, 1.0, api.LENS_MIXED, outp, beta=(1.0, -2.0), stream=stream), 5)
    try:
        import oracle
        rng = np.random.default_rng(8)
        ii, jj = rng.integers(0, MAP_N, 4000), rng.integers(0, MAP_N, 4000)
        dxy = 200.0 / (MAP_N - 1)
        ref = oracle.potential(m, -100.0 + ii * dxy, -100.0 + jj * dxy, 1.0)
        got = outp[0, torch.from_numpy(jj).to(dev), torch.from_numpy(ii).to(dev)].cpu().numpy()
        errs["potential_map"] = {"phi_abs": float(np.max(np.abs(got - ref))),
                                 "phi_range": float(ref.max() - ref.min()),
                                 "frac_of_tolerance": float(np.max(np.abs(got - ref)) /
                                                            (1e-6 * (ref.max() - ref.min()) + 1e-9 * np.abs(ref).max())),
                                 "nodes": 4000}
    except Exception as e:
        errs["potential_map"] = {"error": str(e)}
    ex["potential_map_mixed"] = {"ms": t, "pair_per_s": pairs / (t * 1e-3),
                                 "ops_per_pair": POT_FP32_OPS_PER_PAIR,
                                 "fp32_frac": POT_FP32_OPS_PER_PAIR * pairs / (t * 1e-3)
                                 / (SMS * FP32_LANES * 2.07e9) if POT_FP32_OPS_PER_PAIR else None,
                                 "workload": "potential + Fermat surface, 2048^2 x 1000, LENS_MIXED"}
    del outp
    # the same map with the members' cut radii at 45" (L/L*)^1/2 instead of
    # 8" (L/L*)^1/2: more (point, member) pairs inside a cut radius
    m45 = I.cfg2_model(rcut_star=45.0)
    mid45 = ctx.model_upload(m45)
    t45 = timed(lambda: ctx.hessian_map(mid45, g, 1.0, api.LENS_MIXED, out, stream), 5)
    ex["hessian_map_rcut45"] = {"ms": t45, "pair_per_s": pairs / (t45 * 1e-3),
                                "interp_range_frac": interp_range_fraction(m45, g),
                                "interp_range_frac_rcut8": interp_range_fraction(m, g),
                                "workload": "hessian_map 2048^2 x 1000, members' r_cut = 45\" (L/L*)^1/2"}
    ctx.model_release(mid45)
    out64 = torch.empty((6, MAP_N, MAP_N), dtype=torch.float64, device=dev)
    t = timed(lambda: ctx.hessian_map(mid, g, 1.0, api.LENS_FP64, out64, stream), 1)
    ex["hessian_map_fp64_gpu"] = {"ms": t, "pair_per_s": pairs / (t * 1e-3)}
    del out64
    m1, g1 = I.cfg1_model(), I.grid(256)
    mid1 = ctx.model_upload(m1)
    o1 = torch.empty((2, 256, 256), dtype=torch.float64, device=dev)
    t = timed(lambda: ctx.grad_map(mid1, g1, 0.7, api.LENS_FP64, o1, stream), 50)
    ex["grad_map_fp64_256x10"] = {"ms": t}
    # batched chi2 on the 1000-potential model with its multiple-image
    # constraints (100 sources, 372 images at 5 distance ratios)
    cons = I.load_constraints(os.path.join(ROOT, "tests", "golden", "cfg2_constraints.json"))
    cs = ctx.cset_create(mid, cons, (0, 1))
    P = 4096
    params = torch.tensor(I.perturbed_params(m, (0, 1), P, seed=35), device=dev)
    chi2 = torch.empty(P, dtype=torch.float64, device=dev)
    t_default = timed(lambda: ctx.chi2_source(cs, params, P, 0, chi2, stream), 5)
    cfg, _ = ctx.chi2_autotune(cs, params, P, chi2, stream)
    # one persistent launch per batch, captured once in a CUDA graph and replayed
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    ctx.chi2_source(cs, params, P, 0, chi2, side)
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        ctx.chi2_source(cs, params, P, 0, chi2, side)
    t = timed(lambda: graph.replay(), 20)
    chi2_src_gpu = chi2[:64].cpu().numpy()
    ex["chi2_source"] = {"ms": t, "models_per_s": P / (t * 1e-3), "images": int(cons["img_off"][-1]), "P": P,
                         "ms_default_shape": t_default, "autotuned_shape": cfg, "graph_replay": True,
                         "roofline": leg_roofline(CHI2_SRC_OPS, P / (t * 1e-3), 2.07e9),
                         "workload": "source-plane chi2, 4096 parameter sets, 1000 potentials"}
    # Metropolis sampling on the device: 4096 chains over the two cluster
    # halos' 14 parameters, one step = proposals + batched chi2 + acceptance
    walk = params.clone()
    wchi2 = torch.empty(P, dtype=torch.float64, device=dev)
    ctx.chi2_source(cs, walk, P, 0, wchi2, stream)
    sig = torch.tensor([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1] * 2, dtype=torch.float64, device=dev)
    scratch = torch.empty(16 * P, dtype=torch.float64, device=dev)
    acc = torch.empty(P, dtype=torch.int32, device=dev)
    nsteps = 20
    state = {"k": 0, "acc": 0}

    def mcmc_steps():
        for _ in range(nsteps):
            ctx.mcmc_step(cs, walk, wchi2, P, sig, 2000.0, 2024, state["k"], scratch, acc, stream=stream)
            state["k"] += 1

    t = timed(mcmc_steps, 1) / nsteps
    ctx.mcmc_step(cs, walk, wchi2, P, sig, 2000.0, 2024, state["k"], scratch, acc, stream=stream)
    torch.cuda.synchronize()
    # the same with the members' scaling factors moving too (16 parameters)
    walk16 = torch.cat([params, torch.ones((P, 2), dtype=torch.float64, device=dev)], 1)
    wchi16 = torch.empty(P, dtype=torch.float64, device=dev)
    ctx.chi2_source_scaled(cs, walk16, P, 0, wchi16, stream)
    sig16 = torch.cat([sig, torch.tensor([0.02, 0.05], dtype=torch.float64, device=dev)])
    scratch16 = torch.empty(18 * P, dtype=torch.float64, device=dev)
    t16 = timed(lambda: ctx.mcmc_step(cs, walk16, wchi16, P, sig16, 2000.0, 7, 0, scratch16, acc, stream=stream), 1)
    ctx.cset_scaling_cache(cs, 0.5, 2.0, 32)
    ctx.chi2_source_scaled(cs, walk16, P, 0, wchi16, stream)
    t16c = timed(lambda: ctx.mcmc_step(cs, walk16, wchi16, P, sig16, 2000.0, 7, 1, scratch16, acc, stream=stream), 5)
    ctx.cset_scaling_cache(cs, 0.0, 0.0, 0)
    ex["mcmc_step_scaled_cached"] = {"ms": t16c, "steps_per_s": 1e3 / t16c, "models_per_s": P / (t16c * 1e-3),
                                     "chains": P, "workload": "as mcmc_step_scaled, chi2 from the scaling cache"}
    ex["mcmc_step_scaled"] = {"ms": t16, "steps_per_s": 1e3 / t16, "models_per_s": P / (t16 * 1e-3), "chains": P,
                              "workload": "Metropolis step of 4096 chains over 16 parameters (the members' "
                                          "scaling factors too; chi2 with every static potential per set)"}
    ex["mcmc_step"] = {"ms": t, "steps_per_s": 1e3 / t, "models_per_s": P / (t * 1e-3), "chains": P,
                       "accept_frac_last_step": float(acc.float().mean()),
                       "workload": "Metropolis step of 4096 chains (Philox proposals, source-plane chi2, "
                                   "acceptance), 1000 potentials, temperature 2000"}
    # the same without the static cache: every potential at every image for
    # every set (double-float), the per-model cost when any potential may vary
    t = timed(lambda: ctx.chi2_source_nocache(cs, params, P, 0, chi2, stream), 1)
    nimg = int(cons["img_off"][-1])
    ex["chi2_source_nocache"] = {"ms": t, "models_per_s": P / (t * 1e-3), "P": P,
                                 "pair_per_s": nimg * (N_HALO - 2) * P / (t * 1e-3),
                                 "workload": "source-plane chi2 without the static cache, 4096 sets x 372 images "
                                             "x 1000 potentials, double-float with Hessian"}
    # members' scaling relations free as well: 16 parameters per set, the
    # static sums recomputed per set (double-float)
    p16 = torch.cat([params, torch.tensor(np.random.default_rng(36).uniform(0.8, 1.2, (P, 2)), device=dev)], 1)
    t = timed(lambda: ctx.chi2_source_scaled(cs, p16, P, 0, chi2, stream), 1)
    ex["chi2_source_scaled"] = {"ms": t, "models_per_s": P / (t * 1e-3), "P": P,
                                "pair_per_s": nimg * (N_HALO - 2) * P / (t * 1e-3),
                                "workload": "source-plane chi2 with the members' b0 and r_cut factors free, 4096 "
                                            "sets x 372 images x 1000 potentials, double-float with Hessian"}
    # ... and from the scaling cache: the static sums at 32 Chebyshev nodes
    # of the r_cut factor on [0.5, 2], interpolated per set
    t0 = time.perf_counter()
    ctx.cset_scaling_cache(cs, 0.5, 2.0, 32)
    build_ms = (time.perf_counter() - t0) * 1e3
    t = timed(lambda: ctx.chi2_source_scaled(cs, p16, P, 0, chi2, stream), 5)
    ex["chi2_source_scaled_cached"] = {"ms": t, "models_per_s": P / (t * 1e-3), "P": P, "cache_build_ms": build_ms,
                                       "workload": "as chi2_source_scaled, the static sums interpolated from 32 "
                                                   "Chebyshev nodes of the r_cut factor"}
    Pi = 256
    gi = I.grid(1024)
    chi2i = torch.empty(Pi, dtype=torch.float64, device=dev)
    t = timed(lambda: ctx.chi2_image(cs, gi, params[:Pi], Pi, chi2i, None, stream), 2)
    nf_img = torch.empty((Pi, len(cons["img_off"]) - 1), dtype=torch.int32, device=dev)
    ctx.chi2_image(cs, gi, params[:1], 1, chi2i, nf_img, stream)
    torch.cuda.synchronize()
    chi2_img_gpu, nf_img_gpu = float(chi2i[0]), nf_img[0].cpu().numpy()
    ex["chi2_image"] = {"ms": t, "models_per_s": Pi / (t * 1e-3), "P": Pi,
                        "roofline": leg_roofline(CHI2_IMG_OPS, Pi / (t * 1e-3), 2.07e9),
                        "workload": "image-plane chi2, 1024^2 triangulated grid, 256 parameter sets, 1000 potentials"}
    # request loop: mixed Poisson stream over 8 resident models
    try:
        ex["serving"] = serving_leg(ctx, api, torch)
    except Exception as e:  # keep the line
        ex["serving"] = {"error": str(e)}
    # CPU baseline: the oracle on the host cores, ~15 s of row bands
    try:
        rate, rows, thr = oracle_map_sample(m, g, 15.0)
        ex["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                              "sample": f"{rows} rows x 2048 points x 1000 potentials (FP64 C, OpenMP)"}
    except Exception as e:  # the benchmark line still prints without it
        ex["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                              "sample": f"failed: {e}"}
    try:
        ex["cpu_oracle_other"], ref_src, ref_img, ref_nf = oracle_other_legs(m, g, cons, params.cpu().numpy())
        rel = np.abs(chi2_src_gpu - ref_src) / np.abs(ref_src)
        errs["chi2_source"] = {"rel_max": float(rel.max()), "sets": len(rel), "variant": 0}
        errs["chi2_image"] = {"rel": abs(chi2_img_gpu - ref_img) / abs(ref_img), "sets": 1,
                              "image_counts_equal": bool(np.array_equal(nf_img_gpu, ref_nf)),
                              "grid": "1024^2"}
    except Exception as e:
        ex["cpu_oracle_other"] = {"error": str(e)}
    return ex


def oracle_other_legs(m, g, cons, params):
    """The oracle on the host cores for the other workloads (bounded samples):
    the Hessian map on one core, source-plane chi2 on 64 sets, image-plane
    chi2 on one set of the 1024^2 grid."""
    import oracle
    from paper_2004_06352_gb300 import inputs as I
    out = {}
    thr = oracle.num_threads()
    oracle.set_threads(1)
    try:
        rate, rows, _ = oracle_map_sample(m, g, 3.0)
    finally:
        oracle.set_threads(thr)
    out["hessian_map_1core"] = {"pair_per_s": rate, "cores": 1, "sample": f"{rows} rows x 2048 x 1000"}
    n = 64
    t0 = time.perf_counter()
    ref_src = oracle.chi2_source_batch(m, cons, (0, 1), params[:n], 0)
    dt = time.perf_counter() - t0
    out["chi2_source"] = {"models_per_s": n / dt, "cores": thr, "sample": f"{n} parameter sets"}
    t0 = time.perf_counter()
    ref_img, ref_nf = oracle.chi2_image_batch(m, cons, I.grid(1024), (0, 1), params[:1])
    dt = time.perf_counter() - t0
    out["chi2_image"] = {"models_per_s": 1.0 / dt, "cores": thr, "sample": "1 parameter set, 1024^2 grid"}
    return out, ref_src, float(ref_img[0]), ref_nf[0]


def profile_leg(args):
    """One workload, warmup + steps launches, for profilers."""
    import torch
    from paper_2004_06352_gb300 import build as B
    B.build()
    from paper_2004_06352_gb300 import api
    from paper_2004_06352_gb300 import inputs as I
    dev = torch.device("cuda", 0)
    ctx = api.Context(0)
    m = I.cfg2_model()
    mid = ctx.model_upload(m)
    if args.profile_leg == "map":
        g = I.grid(MAP_N)
        out = torch.empty((6, MAP_N, MAP_N), dtype=torch.float32, device=dev)
        run = lambda: ctx.hessian_map(mid, g, 1.0, api.LENS_MIXED, out)
    elif args.profile_leg == "potential":
        g = I.grid(MAP_N)
        out = torch.empty((2, MAP_N, MAP_N), dtype=torch.float64, device=dev)
        run = lambda: ctx.potential_map(mid, g, 1.0, api.LENS_MIXED, out, beta=(1.0, -2.0))
    else:
        cons = I.load_constraints(os.path.join(ROOT, "tests", "golden", "cfg2_constraints.json"))
        cs = ctx.cset_create(mid, cons, (0, 1))
        P = 256 if args.profile_leg == "chi2_image" else 4096
        params = torch.tensor(I.perturbed_params(m, (0, 1), P, seed=35), device=dev)
        chi2 = torch.empty(P, dtype=torch.float64, device=dev)
        if args.profile_leg == "chi2_source":
            run = lambda: ctx.chi2_source(cs, params, P, 0, chi2)
        elif args.profile_leg == "mcmc":
            # Metropolis steps of 4096 chains (14 parameters)
            ctx.chi2_source(cs, params, P, 0, chi2)
            sig = torch.tensor([0.2, 0.2, 0.005, 0.01, 0.05, 5.0, 0.1] * 2, dtype=torch.float64, device=dev)
            scratch = torch.empty(16 * P, dtype=torch.float64, device=dev)
            state = {"k": 0}

            def run():
                ctx.mcmc_step(cs, params, chi2, P, sig, 2000.0, 5, state["k"], scratch)
                state["k"] += 1
        elif args.profile_leg == "scaled":
            # the members' scaling factors free: recomputed sums, then the cache
            p16 = torch.cat([params, torch.full((P, 2), 1.05, dtype=torch.float64, device=dev)], 1)
            ctx.chi2_source_scaled(cs, p16, P, 0, chi2)
            ctx.cset_scaling_cache(cs, 0.5, 2.0, 32)
            run = lambda: ctx.chi2_source_scaled(cs, p16, P, 0, chi2)
        else:
            gi = I.grid(1024)
            run = lambda: ctx.chi2_image(cs, gi, params, P, chi2)
    for _ in range(args.warmup + args.steps):
        run()
    ctx.wait()
    ctx.close()


def serving_leg(ctx, api, torch):
    """Capacity (closed loop, <= 8 outstanding) and p50/p99 latency of Poisson
    streams at 50/80/95 % of capacity: 60 % Hessian maps 512^2-8192^2 on
    models of 10-2000 potentials, 40 % source-plane chi2 of 16-4096 sets;
    plus the same requests (maps <= 2048^2) served by the plain FP64 form."""
    from paper_2004_06352_gb300 import serving as S
    out = {}
    models = S.resident_models(8, seed=11)
    sess = S.Session(ctx, models)
    srv = api.Server(ctx, slots=4, pool_bytes=12 << 30)
    pool = S.PinnedPool()
    # page-lock the result buffers before timing (on demand, page-locking a
    # 1.6 GB 8192^2 result blocks the submitting loop for a good part of a
    # second, which an open stream near capacity never recovers from)
    for side in S.MAP_SIDES:
        for _ in range(8 if side == 8192 else 12 if side == 4096 else 16):
            pool.give(torch.empty((6, side, side), dtype=torch.float32, pin_memory=True))
    for _ in range(48):
        pool.give(torch.empty((S.PinnedPool.VEC_CAP,), dtype=torch.float64, pin_memory=True))
    warm = S.mixed_requests(8, seed=12, n_models=8, sides=(512, 1024))
    S.run_stream(srv, sess, warm, pool=pool, max_outstanding=8, keep_results=False)
    # one request list (400 requests) for the capacity and every load level;
    # the load levels share one Poisson draw, scaled to each rate, so they
    # differ only in rate and not in the shape of their bursts
    reqs = S.mixed_requests(400, seed=13, n_models=8)
    lat, wall, _, _ = S.run_stream(srv, sess, reqs, pool=pool, max_outstanding=8, keep_results=False)
    cap = len(reqs) / wall
    out["capacity_req_per_s"] = cap
    out["closed_loop"] = S.percentiles(lat)
    for frac in (0.5, 0.8, 0.95):
        arr = S.poisson_arrivals(len(reqs), frac * cap, seed=15)
        miss0 = pool.misses
        lat, wall, _, _ = S.run_stream(srv, sess, reqs, arr, pool=pool, keep_results=False)
        out[f"load_{int(100 * frac)}"] = dict(S.percentiles(lat), offered_req_per_s=frac * cap,
                                               served_req_per_s=len(reqs) / wall, n=len(reqs),
                                               pinned_on_demand=pool.misses - miss0)
    srv.close()
    # same small-map requests through the mixed and the plain FP64 forms
    small = S.mixed_requests(24, seed=14, n_models=8, sides=(512, 1024, 2048))
    res = {}
    for name, prec, rr in (("mixed", api.LENS_MIXED, api.LENS_REPAIR_RATIO_DEFAULT),
                           ("mixed_no_repair", api.LENS_MIXED, 0.0), ("fp64", api.LENS_FP64, 0.0)):
        ctx.set_repair_ratio(rr)
        s2 = S.Session(ctx, models, precision=prec)
        srv = api.Server(ctx, slots=4, pool_bytes=4 << 30)
        S.run_stream(srv, s2, small[:4], pool=pool, max_outstanding=8, keep_results=False)  # warm
        lat, wall, _, _ = S.run_stream(srv, s2, small, pool=pool, max_outstanding=8, keep_results=False)
        res[name] = dict(S.percentiles(lat), req_per_s=len(small) / wall)
        srv.close()
    ctx.set_repair_ratio(api.LENS_REPAIR_RATIO_DEFAULT)
    out["mixed_vs_fp64_same_requests"] = res
    out["workload"] = ("Poisson mix: 60% Hessian maps side 512-8192 (uniform over powers of 2), 8 resident models "
                       "of 10-2000 potentials; 40% source-plane chi2 with 16-4096 sets; 4 slots, 12 GiB pool")
    return out


if __name__ == "__main__":
    main()
