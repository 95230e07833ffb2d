"""Benchmark of the subcycled M1 radiation update on GB300.

Workload (throughput configuration): 512^3 periodic grid, radiation (E, Fx, Fy, Fz) plus frozen gas
(rho, T, vx, vy, vz) with a seeded lognormal density (sigma_ln rho = 1), absorption coefficients
proportional to rho (k = 512 rho), gas speeds v ~ N(0, (0.001 c)^2), isotropic random F with
|F| <= 0.5 cE, FULL energy exchange and O(beta tau) terms,
c = 10, chat = 1, CFL 0.4.  One step = one call of rhd_radiation_subcycle with 100 subcycles, i.e. the
whole hot path (every per-subcycle stage) over the grid.  Headline: the split-precision path; the plain
FP64 path is measured alongside (4 subcycles per step, same rate unit).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on the host cores on a bounded
sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "radiation cell-updates/s per subcycle (FP64 vs FP32/FP64 split) and % HBM roofline"
UNIT = "cell-updates/s"
# algorithmic bytes per cell-update of the throughput workload (FULL exchange, beta tau on, opacity law
# k = 512 rho evaluated in registers): U^m read + U^{m+1} write 64 B, T read + write 16 B, rho and v read
B_ALG = {"fp64": 64 + 16 + 8 + 24, "split": 64 + 16 + 4 + 12}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--launch", default="auto",
                    help="split-path launch configuration: 'auto' (autotune before timing) or "
                         "VARIANT:TXxTY:zZCHUNK:STAGING, e.g. twopass:32x8:z32:cpasync")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--n-sub", type=int, default=100)
    ap.add_argument("--fp64-n-sub", type=int, default=4)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (1D wave, 2D source, 3D shell, ensemble)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="throughput", choices=["throughput", "ensemble", "marshak"],
                    help="throughput: one 512^3 grid (the headline); ensemble: 64 independent grids of "
                         "32^3..128^3, one persistent launch per subcycle, against per-grid plain launches; "
                         "marshak: the paper's timing benchmark, the 1D non-equilibrium Marshak wave to "
                         "tau = 1, 10, 100 on N = 32 .. 2048 cells")
    ap.add_argument("--marshak-cpu-cells", type=float, default=3e5,
                    help="marshak: time the oracle only on runs of at most this many cell-updates")
    ap.add_argument("--marshak-sizes", default="32,64,128,256,512,1024,2048",
                    help="marshak: the cell counts N (comma-separated)")
    ap.add_argument("--marshak-taus", default="1,10,100", help="marshak: the optical times tau (comma-separated)")
    ap.add_argument("--n-grids", type=int, default=64)
    ap.add_argument("--traffic-from", default=None,
                    help="write profiles/traffic.json from this ncu raw CSV (measured at --N, scaled to 512^3; "
                         "--launch names the configuration) and exit")
    ap.add_argument("--fp64-ops-from", default=None,
                    help="write profiles/fp64_ops.json (FP64 instructions per cell-update of the FP64 fused "
                         "kernel) from this ncu raw CSV of one launch at --N and exit")
    ap.add_argument("--ens-n-sub", type=int, default=50, help="subcycles per step of the ensemble workload")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def cpu_baseline(case, seconds, n_cells_box=64):
    """Oracle (plain C, FP64, OpenMP over cells) on bounded boxes of the same grid, one subcycle each."""
    from oracle import oracle as orc

    N = case["desc"]["n"][0]
    g = np.random.default_rng(1)
    t0 = time.perf_counter()
    cells = 0
    boxes = 0
    while True:
        lo = [int(v) for v in g.integers(0, N - n_cells_box, size=3)]
        hi = [v + n_cells_box for v in lo]
        orc.subcycle_box(case, lo, hi)
        cells += n_cells_box ** 3
        boxes += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": cells / el, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"{boxes} boxes of {n_cells_box}^3 cells of the {N}^3 grid, one subcycle each "
                      f"({el:.1f} s of CPU work)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import build_oracle
    from paper_1306_0010_gb300 import workloads as wl

    build_oracle.build()
    case = wl.config4(N=args.N, n_sub=args.n_sub)
    per_step = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(case, per_step / 4)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(case, per_step))
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[0], value=v)
    cells_per_step = args.N ** 3 * args.n_sub
    # each timed step is a bounded sample (boxes of the grid); ms_per_step is that rate extrapolated to a
    # whole step of the workload (N^3 cells x n_sub subcycles), not a time the run took
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cells_per_step / v,
            "ms_per_step_kind": "extrapolated from the timed samples to one step of the workload",
            "sample_seconds_per_step": per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, "fp64"),
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# the sources the split path's kernels (predictor, corrector) are compiled from
SPLIT_KERNEL_SOURCES = ("dfloat.cuh", "fp_convert.cuh", "k_split.cu", "rhd_internal.h", "subcycle.cuh",
                        "subcycle_pair.cuh", "subcycle_twopass.cuh")


def kernel_source_hash(sources=SPLIT_KERNEL_SOURCES):
    """SHA-256 over the code of a path's kernels (comments and whitespace removed): ncu figures
    recorded for other kernel code are stale."""
    import hashlib
    import re

    d = os.path.join(ROOT, "paper_1306_0010_gb300", "csrc")
    h = hashlib.sha256()
    for name in sources:
        text = open(os.path.join(d, name), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(name.encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def record_traffic(csv_path, measured_N, target_N, launch_spec):
    """Write profiles/traffic.json from an `ncu --page raw --csv` export: DRAM bytes per launch of each
    split kernel, scaled from measured_N^3 to target_N^3 cells (traffic grows with the cell count)."""
    import csv

    names = {"predictor_kernel": "twopass_predictor_split", "corrector_kernel": "twopass_corrector_split"}
    rows = list(csv.reader(open(csv_path)))
    first = next(i for i, r in enumerate(rows) if "Kernel Name" in r)  # ncu's own log lines come first
    rows = rows[first:]
    hdr, units = rows[0], rows[1]
    scale = (target_N / measured_N) ** 3
    out = {"note": f"dram__bytes_read.sum + dram__bytes_write.sum per launch, ncu at {measured_N}^3, scaled to "
                   f"{target_N}^3 by the cell count", "source_sha256": kernel_source_hash()}
    unit_mult = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    for r in rows[2:]:
        kname = r[hdr.index("Kernel Name")]
        key = next((v for k, v in names.items() if k in kname), None)
        if key is None:
            continue
        b = 0.0
        for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            j = hdr.index(m)
            b += float(r[j].replace(",", "")) * unit_mult[units[j]]
        out[key] = {"N": target_N, "launch": launch_spec, "bytes_per_launch": b * scale, "measured_N": measured_N,
                    "measured_bytes_per_cell": b / measured_N ** 3}
    path = os.path.join(ROOT, "profiles", "traffic.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


# the sources the FP64 fused kernel is compiled from
FP64_KERNEL_SOURCES = ("dfloat.cuh", "fp_convert.cuh", "k_fp64.cu", "rhd_internal.h", "subcycle.cuh",
                       "subcycle_pair.cuh", "subcycle_twopass.cuh")
# FP64 issue peak from unit counts and the maximum SM clock: 152 SMs x 2 FP64 operations per cycle (the
# ncu peak of sm__sass_thread_inst_executed_op_dfma_pred_on is 304 per cycle) x 2.07 GHz
FP64_PEAK_TOPS = 152 * 2 * 2.07e9 / 1e12


def record_fp64_ops(csv_path, N):
    """Write profiles/fp64_ops.json from an `ncu --page raw --csv` export of one FP64 fused-kernel launch
    over N^3 cells: thread-level dadd + dfma + dmul instructions per cell-update."""
    import csv

    rows = list(csv.reader(open(csv_path)))
    first = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr, rows = rows[first], rows[first + 2:]
    r = next(r for r in rows if "subcycle_kernel<double" in r[hdr.index("Kernel Name")])
    ops = {}
    for op in ("dadd", "dfma", "dmul"):
        ops[op] = float(r[hdr.index(f"smsp__sass_thread_inst_executed_op_{op}_pred_on.sum")].replace(",", "")) / N ** 3
    out = {"note": f"FP64 thread instructions per cell-update of the FP64 fused kernel, ncu at {N}^3 (one launch)",
           "source_sha256": kernel_source_hash(FP64_KERNEL_SOURCES), "N": N, "per_cell_update": ops,
           "fp64_ops_per_cell_update": sum(ops.values())}
    with open(os.path.join(ROOT, "profiles", "fp64_ops.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


def fp64_pipe_roofline(rate):
    """The FP64 path against the FP64 issue peak: its kernel's FP64 instructions per cell-update (ncu,
    profiles/fp64_ops.json, dropped when the kernel's sources have changed since) times the rate."""
    path = os.path.join(ROOT, "profiles", "fp64_ops.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != kernel_source_hash(FP64_KERNEL_SOURCES):
        return None
    ops = float(rec["fp64_ops_per_cell_update"])
    achieved = ops * rate / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TOPS, "unit": "T FP64 instr/s",
            "frac": achieved / FP64_PEAK_TOPS, "fp64_ops_per_cell_update": ops,
            "peak_kind": "derived: 152 SMs x 2 FP64 operations per cycle x 2.07 GHz"}


def launch_key(launch):
    return f"{launch['variant']}:{launch['tile'][0]}x{launch['tile'][1]}:z{launch['z_chunk']}:{launch['staging']}"


def workload_config(args, precision):
    return {"workload": f"3D throughput run, {args.N}^3 periodic SoA grid, lognormal rho (sigma_ln rho = 1), "
                        f"v ~ N(0, (0.001 c)^2), k = 512 rho, |F| <= 0.5 cE, FULL exchange, beta tau on, "
                        f"c = 10, chat = 1",
            "N": args.N, "n_sub_per_step": args.n_sub, "precision": precision,
            "l2": "inputs larger than L2 (1.07 GB per FP64 field)"}


def max_over_ranks(local_ms, dist=None, device=None):
    """Slowest rank's time (every rank gets it); local_ms itself on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_ms)
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells, n_sub, steps, world_size, max_ms):
    """Cell-updates of all ranks (each advances its own grid of `cells` cells) over the slowest rank's time."""
    return cells * n_sub * steps * world_size / (max_ms * 1e-3)


def parse_launch(spec):
    v, t, z, stg = spec.split(":")
    tx, ty = (int(x) for x in t.split("x"))
    return {"variant": v, "tile": (tx, ty), "z_chunk": int(z.lstrip("z")), "staging": stg}


def time_rsla(torch, g, case, stream, hbm_peak, reps=5):
    """The reduced-speed-of-light reductions on the same grid (inputs larger than L2): CUDA events on
    the library's stream around each call (the call synchronises after its kernels and an 8-byte
    copy).  Algorithmic bytes: v_max reads rho, T, E and each velocity component and kF array the
    grid has; tau_max reads kF (or rho for the opacity law) once per active axis."""
    f = case["fields"]
    cells = int(np.prod(f["rho"].shape))
    n_v = sum(f.get(k) is not None for k in ("vx", "vy", "vz"))
    has_kF = f.get("kF") is not None
    n_axes = sum(int(v) > 1 for v in case["desc"]["n"])
    out = {}
    for name, call, bpc in (("max_signal_speed", g.max_signal_speed, 8 * (3 + n_v + has_kF)),
                            ("max_optical_depth", g.max_optical_depth, 8 * n_axes)):
        call()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        for r in range(reps):
            ev[2 * r].record(stream)
            call()
            ev[2 * r + 1].record(stream)
        stream.synchronize()
        ms = min(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(reps))
        gbs = bpc * cells / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes_per_cell": bpc, "achieved_gbs": gbs, "frac": gbs / hbm_peak}
    return out


def time_gas(torch, g, case, stream, hbm_peak, peak_kind, reps=3):
    """The gas step (Section 3.1 step 3) and its source correction (step 6) on the same grid, after the
    radiation legs: dt_gas = 0.1 min(dx) (a Courant number near 0.2 for this gas), one untimed step
    (scratch allocation), then `reps` timed (step, correction) pairs with CUDA events on the library's
    stream and the kernel timer.  Rate: interior cells advanced per second of (step + correction)."""
    dx = min(case["desc"]["dx"][d] for d in range(3) if case["desc"]["n"][d] > 1)
    dt = 0.1 * dx
    cells = int(np.prod(case["fields"]["rho"].shape))
    g.gas_step(dt)
    g.gas_correct()
    stream.synchronize()
    g.kernel_times()  # discard
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for r in range(reps):
        g.gas_step(dt)
        g.gas_correct()
        ev[r + 1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[-1]) / reps
    kt = g.kernel_times()
    st = g.get_stats(allow_nonfinite=True)
    return {"value": cells / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_gas_step": ms, "dt_gas": dt,
            "kernels": kt, "roofline": kernel_roofline(kt, hbm_peak, peak_kind),
            "gpu_launches": sum(v["launches"] for v in kt.values()) // reps,
            "gas_energy_floors": st["gas_energy_floors"], "gas_nonfinite": st["gas_nonfinite"]}


def time_path(torch, rhd, case, precision, n_sub, steps, warmup, stream, tune=True, launch_spec="auto",
              rsla_peak=None, peak_kind="measured"):
    """Device-resident run: autotune the launch configuration (untimed), warm up, then time `steps`
    calls of n_sub subcycles with CUDA events on the library's stream.  The kernel timer brackets
    every kernel of the timed region with events on the same stream (plain launches)."""
    desc = dict(case["desc"], precision=precision)
    g = rhd.Grid(desc, stream=stream.cuda_stream)
    f = case["fields"]
    dev = {k: (None if f[k] is None else torch.from_numpy(f[k]).to("cuda")) for k in f}
    with torch.cuda.stream(stream):
        g.set_gas_state(dev["rho"], dev["T"], dev["vx"], dev["vy"], dev["vz"], dev["kP"], dev["kF"], dev["j"])
        g.set_moments(dev["E"], dev["Fx"], dev["Fy"], dev["Fz"])
    stream.synchronize()
    tuning = None
    if tune and launch_spec != "auto":
        g.set_launch_config(parse_launch(launch_spec))
    elif tune:
        chosen, table = g.autotune(case["chat"], case["dt"], reps=3)
        tuning = {"chosen": chosen, "candidates": table}
    launch = g.launch_config()
    g.set_kernel_timing(True)
    for _ in range(warmup):
        g.radiation_subcycle(n_sub, case["chat"], case["dt"])
    stream.synchronize()
    g.kernel_times()  # discard the warm-up interval
    g.reset_stats()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for s in range(steps):
        g.radiation_subcycle(n_sub, case["chat"], case["dt"])
        ev[s + 1].record(stream)
    stream.synchronize()
    per_step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    kt = g.kernel_times()
    st = g.get_stats(allow_nonfinite=True)
    g.set_kernel_timing(False)
    rsla = time_rsla(torch, g, case, stream, rsla_peak) if rsla_peak else None
    if rsla is not None:
        g.set_kernel_timing(True)
        rsla["gas_step"] = time_gas(torch, g, case, stream, rsla_peak, peak_kind)
        g.set_kernel_timing(False)
    g.close()
    del dev
    return total_ms, per_step_ms, st, kt, launch, tuning, rsla


# FP32 peak from unit counts and the maximum SM clock: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def alu_roofline(rate):
    """The split path against the FP32 arithmetic peak: the oracle's operation count per cell-update
    (add + mul + div + sqrt of the plain FP64 algorithm, from its counting build) times the rate."""
    path = os.path.join(ROOT, "profiles", "opcounts.json")
    if not os.path.exists(path):
        return None
    ops = float(json.load(open(path))["arith_per_cell_update"])
    achieved = ops * rate / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "ops_per_cell_update": ops,
            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz"}


def kernel_roofline(kt, peak, peak_kind):
    """Roofline of the kernel with the largest share of the timed region: algorithmic bytes of one
    launch over its mean event-measured duration."""
    name = max(kt, key=lambda k: kt[k]["total_ms"])
    k = kt[name]
    mean_ms = k["total_ms"] / k["launches"]
    achieved = k["alg_bytes_per_launch"] / (mean_ms * 1e-3) / 1e9
    total = sum(v["total_ms"] for v in kt.values())
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "peak_kind": peak_kind, "kernel": name, "launch_ms": mean_ms,
            "alg_bytes_per_launch": k["alg_bytes_per_launch"], "share_of_kernel_time": k["total_ms"] / total}


def time_e2e(torch, rhd, case, precision, n_sub, steps, warmup, launch_spec="auto"):
    """Same metric through the public API with host (pinned) buffers: per step, H2D of the moments and
    gas state, the subcycles, D2H of the moments and temperature.  Two grids on two streams take the
    steps in turn, so one step's copies run while the other grid computes (the upload and the
    subcycles are asynchronous on a grid's stream; reading the results waits for that grid only).  The
    launch configuration is the autotuner's (RHD_FLAG_AUTOTUNE: reused from the device-resident run's
    tuning of the same shape) or the one given."""
    desc = dict(case["desc"], precision=precision, flags=rhd.FLAG_AUTOTUNE if launch_spec == "auto" else 0)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    grids = [rhd.Grid(desc, stream=st.cuda_stream) for st in streams]
    if launch_spec != "auto":
        for g in grids:
            g.set_launch_config(parse_launch(launch_spec))
    f = case["fields"]
    pin = {k: (None if f[k] is None else torch.from_numpy(f[k]).pin_memory()) for k in f}
    outs = [[torch.empty(f["E"].shape, dtype=torch.float64).pin_memory() for _ in range(5)] for _ in grids]
    h2d = sum(v.numel() * 8 for k, v in pin.items() if v is not None and k in
              ("E", "Fx", "Fy", "Fz", "rho", "T", "vx", "vy", "vz", "kP", "kF", "j"))
    d2h = sum(o.numel() * 8 for o in outs[0])

    def issue(s):  # step s: its inputs in, its subcycles (asynchronous on its grid's stream)
        g = grids[s % 2]
        g.set_gas_state(pin["rho"], pin["T"], pin["vx"], pin["vy"], pin["vz"], pin["kP"], pin["kF"], pin["j"])
        g.set_moments(pin["E"], pin["Fx"], pin["Fy"], pin["Fz"])
        g.radiation_subcycle(n_sub, case["chat"], case["dt"])

    def read(s):  # step s: its results out (waits for its grid's stream)
        g, o = grids[s % 2], outs[s % 2]
        g.get_moments(o[0], o[1], o[2], o[3])
        g.get_gas_state(o[4])

    for s in range(max(warmup, 2)):  # both grids warm (module loading, tuning, graph capture)
        issue(s)
        read(s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    issue(0)
    for s in range(steps):
        if s + 1 < steps:
            issue(s + 1)
        read(s)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    for g in grids:
        g.close()
    return el, h2d, d2h


def ensemble_workload_config(args, cases):
    sizes = sorted({c["desc"]["n"][0] for c in cases})
    return {"workload": f"ensemble of {len(cases)} independent 3D grids, N drawn from {sizes}, outflow, "
                        f"Gaussian source j with L ~ logU(1e-2, 1e2), uniform opacity tau ~ logU(0.1, 1e3), "
                        f"FULL exchange, theta = 1, c = 10, chat = 1, dt = 0.4 dx / chat per grid",
            "n_grids": len(cases), "cells": sum(int(np.prod(c["desc"]["n"])) for c in cases),
            "n_sub_per_step": args.n_sub, "l2": "inputs larger than L2"}


def time_ensemble(torch, rhd, cases, precision, n_sub, steps, warmup, stream):
    """One persistent launch per subcycle over all grids (tile-to-grid work queue), n_sub subcycles per
    call replayed from a CUDA graph; z chunk autotuned first (untimed)."""
    descs = [dict(c["desc"], precision=precision) for c in cases]
    ens = rhd.Ensemble(descs, stream=stream.cuda_stream)
    for i, c in enumerate(cases):
        ens.load_case(i, c)
    dts = [c["dt"] for c in cases]
    chosen, _ = ens.autotune(1.0, dts, reps=3)
    for _ in range(warmup):
        ens.subcycle(n_sub, 1.0, dts)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ens.subcycle(n_sub, 1.0, dts)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    # kernel timer over one more step (plain launches) for the roofline of the ensemble kernel
    ens.set_kernel_timing(True)
    ens.subcycle(n_sub, 1.0, dts)
    kt = ens.kernel_times()
    st = ens.get_stats(allow_nonfinite=True)
    ens.close()
    return ms, chosen, kt, st


def time_per_grid(torch, rhd, cases, precision, n_sub, steps, warmup, stream):
    """Baseline: each grid its own context, its n_sub subcycles as plain launches (no graph), one grid
    after the other on one stream."""
    grids = []
    for c in cases:
        g = rhd.Grid(dict(c["desc"], precision=precision, flags=rhd.FLAG_NO_GRAPH), stream=stream.cuda_stream)
        g.load_case(c)
        grids.append((g, c["dt"]))
    for _ in range(warmup):
        for g, dt in grids:
            g.radiation_subcycle(n_sub, 1.0, dt)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for g, dt in grids:
            g.radiation_subcycle(n_sub, 1.0, dt)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    for g, _ in grids:
        g.close()
    return ms


# ----------------------------------------------------------------------------- the other configurations

def _grid_run(torch, rhd, case, n_sub, stream, precision=None, flags=0):
    """One timed call of n_sub subcycles (after one untimed warm-up call of the same length on a copy of
    the state); returns (ms, moments, T, stats)."""
    desc = dict(case["desc"], flags=flags)
    if precision is not None:
        desc["precision"] = precision
    g = rhd.Grid(desc, stream=stream.cuda_stream)
    g.load_case(case)
    g.radiation_subcycle(n_sub, case["chat"], case["dt"])  # warm-up (graph capture, module loading)
    g.load_case(case)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.radiation_subcycle(n_sub, case["chat"], case["dt"])
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    out = g.get_moments()
    T = g.get_gas_state()
    st = g.get_stats(allow_nonfinite=True)
    g.close()
    return ms, out, T, st


def run_config1(torch, rhd, wl, stream):
    """1D radiation linear wave (N = 512, periodic, chat = c = 10, CFL 0.4, 1000 subcycles, FP64) at
    optical depths 0.01, 1, 100 per wavelength: the complex frequency measured from the k = 2 pi Fourier
    amplitude of dE against the dispersion relation omega^2 + i chat k_F omega - chat^2 k^2 / 3 = 0."""
    res = {}
    for tau in (0.01, 1.0, 100.0):
        case = wl.config1(tau=tau, mode="equilibrium", N=512, n_sub=1000)
        ms, out, _, st = _grid_run(torch, rhd, case, 1000, stream)
        N = case["desc"]["n"][0]
        x = (np.arange(N) + 0.5) / N
        k = case["k"]
        a0 = np.mean((case["fields"]["E"][0, 0] - 1.0) * np.exp(-1j * k * x)) * 2
        a1 = np.mean((out["E"][0, 0] - 1.0) * np.exp(-1j * k * x)) * 2
        w = 1j * np.log(a1 / a0) / (1000 * case["dt"])
        w_ex = case["omega"]
        res[f"tau_{tau:g}"] = {
            "cell_updates_per_s": N * 1000 / (ms * 1e-3), "ms_per_subcycle": ms / 1000,
            "omega_measured": [float(w.real), float(w.imag)], "omega_relation": [float(w_ex.real), float(w_ex.imag)],
            "phase_speed_rel_error": (abs(w.real - w_ex.real) / abs(w_ex.real)) if abs(w_ex.real) > 0 else None,
            "damping_rel_error": abs(w.imag - w_ex.imag) / abs(w_ex.imag),
            "n_nonfinite": st["n_nonfinite"]}
    return {"workload": "1D radiation linear wave, N = 512 periodic, chat = c = 10, CFL 0.4, 1000 subcycles, FP64, "
                        "EQUILIBRIUM mode, theta = 0.51, dE = 1e-6 cos(2 pi x) on the eigenmode",
            "note": "latency-bound (512 cells): cell-updates/s only", "runs": res}


def run_config2(torch, rhd, wl, stream):
    """2D concentrated source (256^2 on [-1, 1]^2, outflow, Gaussian j of width 0.05 with L = 1, k_F = 1000
    inside r < 0.1 and 0.1 outside, chat = c = 1, 2000 subcycles, FP64): the luminosity through circles
    (the azimuthal mean of F.r_hat times 2 pi r) against L, and realizability fixes."""
    case = wl.config2(N=256, n_sub=2000)
    ms, out, _, st = _grid_run(torch, rhd, case, 2000, stream)
    X, Y, _ = wl.cell_centres(case["desc"], x0=(-1.0, -1.0, 0.0))
    r = np.sqrt(X ** 2 + Y ** 2)[0]
    Fr = ((out["Fx"] * X + out["Fy"] * Y) / np.where(r > 0, r, 1))[0]
    lum = {}
    for r0 in (0.2, 0.3, 0.45, 0.6, 0.75, 0.9):
        ring = np.abs(r - r0) < 0.5 * case["desc"]["dx"][0]
        lum[f"r_{r0:g}"] = float(Fr[ring].mean() * 2 * np.pi * r0 / case["L"])
    g = np.sqrt(out["Fx"] ** 2 + out["Fy"] ** 2) / case["desc"]["c"]
    return {"workload": "2D concentrated source, 256^2 on [-1, 1]^2, outflow, Gaussian j (sigma 0.05, L = 1), "
                        "k_F = 1000 (r < 0.1) / 0.1, chat = c = 1, 2000 subcycles, FP64, EQUILIBRIUM",
            "cell_updates_per_s": 256 * 256 * 2000 / (ms * 1e-3), "ms_per_subcycle": ms / 2000,
            "luminosity_over_L": lum, "realizability_fixes": st["n_realizability_fix"],
            "max_G_over_E": float(np.max(g / out["E"])), "n_nonfinite": st["n_nonfinite"]}


def run_config3(torch, rhd, wl, stream, hbm_peak, n_cycles=20, n_sub=25):
    """3D dusty shell (256^3, outflow, shell rho 100 with tau 10, Gaussian luminosity, FULL exchange, beta
    tau on, chat = 50 v_max, c = 10 chat), the coupled run: n_cycles whole Section 3.1 cycles (gas step,
    n_sub radiation subcycles, source correction; Delta t_gas = n_sub radiation steps, gas Courant number
    0.2) on the split and the FP64 path, and the split path's normwise L1 / L-infinity errors against the
    FP64 path (which the parity tests hold to the oracle at 1e-12, whole cycles included)."""
    case = wl.config3(N=256, n_sub=n_sub)
    cells = 256 ** 3
    dt_gas = n_sub * case["dt"]
    out, res = {}, {}
    for prec in ("split", "fp64"):
        g = rhd.Grid(dict(case["desc"], precision=prec), stream=stream.cuda_stream)
        g.load_case(case)
        g.gas_cycle(case["chat"], dt_gas=dt_gas)  # warm-up (graph capture, scratch), then from the start
        g.load_case(case)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        subs = 0
        for _ in range(n_cycles):
            subs += g.gas_cycle(case["chat"], dt_gas=dt_gas)[1]
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        mom, gas, st = g.get_moments(), g.get_gas(), g.get_stats(allow_nonfinite=True)
        g.close()
        out[prec] = dict(mom, **gas)
        res[prec] = {"cycles": n_cycles, "subcycles": subs, "ms": ms,
                     "radiation_cell_updates_per_s": cells * subs / (ms * 1e-3),
                     "ms_per_cycle": ms / n_cycles, "n_nonfinite": st["n_nonfinite"],
                     "gas_nonfinite": st["gas_nonfinite"], "gas_energy_floors": st["gas_energy_floors"],
                     "realizability_fixes": st["n_realizability_fix"]}
    ref, sp = out["fp64"], out["split"]
    sE = float(np.max(np.abs(ref["E"])))
    sv = float(np.max(np.sqrt(ref["vx"] ** 2 + ref["vy"] ** 2 + ref["vz"] ** 2)))
    err = {}
    for k, sc in (("E", sE), ("Fx", case["desc"]["c"] * sE), ("Fy", case["desc"]["c"] * sE),
                  ("Fz", case["desc"]["c"] * sE), ("rho", float(np.max(ref["rho"]))), ("vx", sv), ("vy", sv),
                  ("vz", sv), ("T", float(np.max(np.abs(ref["T"]))))):
        d = np.abs(sp[k] - ref[k]) / sc
        err[k] = {"L1": float(np.mean(d)), "Linf": float(np.max(d))}
    return {"workload": "3D dusty shell, 256^3, outflow, shell 0.3 <= r <= 0.35 with rho 100 (tau 10), Gaussian "
                        "luminosity (sigma 2 dx, L = 1), FULL exchange, beta tau on, chat = 50 v_max, c = 10 chat, "
                        f"gamma = 5/3; {n_cycles} gas cycles x {n_sub} radiation subcycles",
            "split": res["split"], "fp64": res["fp64"],
            "split_speedup": res["fp64"]["ms"] / res["split"]["ms"],
            "split_error_vs_fp64_path": err}


def run_far_from_equilibrium(torch, rhd, case, launch, stream, relaxed_corrector_ms, n_sub=3):
    """The headline's grid and launch configuration with the radiation 100 times below the gas's
    equilibrium value (E and F of the throughput workload scaled by 0.01, so the gas-to-radiation energy
    ratio K = e / ((c/chat) E) reaches several hundred in dense cells): every cell's energy exchange
    starts far from equilibrium, the regime where its FP32 Newton seed takes the most iterations.  The
    corrector's mean time over the first n_sub subcycles, against its time on the relaxed state the
    headline measures."""
    f = dict(case["fields"])
    for k in ("E", "Fx", "Fy", "Fz"):
        f[k] = 0.01 * f[k]
    far = dict(case, fields=f)
    g = rhd.Grid(dict(case["desc"], precision="split", flags=rhd.FLAG_NO_GRAPH), stream=stream.cuda_stream)
    g.set_launch_config({k: launch[k] for k in ("variant", "tile", "z_chunk", "staging")})
    g.load_case(far)
    g.radiation_subcycle(1, case["chat"], case["dt"])  # module loading
    g.load_case(far)
    g.reset_stats()
    g.set_kernel_timing(True)
    g.radiation_subcycle(n_sub, case["chat"], case["dt"])
    g.synchronize()
    kt = g.kernel_times()
    st = g.get_stats(allow_nonfinite=True)
    g.close()
    corr = next((v for k, v in kt.items() if "corrector" in k), None)
    pred = next((v for k, v in kt.items() if "predictor" in k), None)
    out = {"workload": "the throughput workload with E and F scaled by 0.01 (radiation far below equilibrium), "
                       f"first {n_sub} subcycles", "n_sub": n_sub,
           "newton_iter_max": st["newton_iter_max"], "n_newton_fallback": st["n_newton_fallback"],
           "n_theta_fallback": st["n_theta_fallback"], "n_nonfinite": st["n_nonfinite"]}
    if corr:
        ms = corr["total_ms"] / corr["launches"]
        out.update(corrector_ms=ms, relaxed_corrector_ms=relaxed_corrector_ms,
                   corrector_cost_ratio=ms / relaxed_corrector_ms if relaxed_corrector_ms else None)
    if pred:
        out["predictor_ms"] = pred["total_ms"] / pred["launches"]
    return out


def run_config5(torch, rhd, wl, stream, hbm_peak, peak_kind, steps=3, warmup=1):
    """Batched ensemble: 64 grids of sizes drawn from {32, 48, 64, 96, 128}^3, one persistent launch (pair)
    per subcycle from a 50-subcycle CUDA graph, split (50 subcycles) and FP64 (10), against per-grid
    plain launches."""
    cases = wl.config5(n_grids=64, n_sub=50, precision="split")
    cells = sum(int(np.prod(c["desc"]["n"])) for c in cases)
    res = {"workload": "ensemble of 64 independent 3D grids, N from {32, 48, 64, 96, 128}, outflow, Gaussian j "
                       "with L ~ logU(1e-2, 1e2), uniform tau ~ logU(0.1, 1e3), FULL, theta = 1, c = 10 chat",
           "cells": cells}
    for prec, ns in (("split", 50), ("fp64", 10)):
        ms, chosen, kt, st = time_ensemble(torch, rhd, cases, prec, ns, steps, warmup, stream)
        base_ms = time_per_grid(torch, rhd, cases, prec, ns, max(1, steps - 1), 1, stream)
        res[prec] = {"n_sub_per_step": ns, "value": cells * ns * steps / (ms * 1e-3),
                     "per_grid_plain_launches": cells * ns * max(1, steps - 1) / (base_ms * 1e-3),
                     "launch": chosen, "roofline": kernel_roofline(kt, hbm_peak, peak_kind),
                     "n_nonfinite": st["n_nonfinite"]}
        res[prec]["speedup_vs_per_grid"] = res[prec]["value"] / res[prec]["per_grid_plain_launches"]
    return res


def run_marshak(args):
    """Section 4.2's benchmark: wall-clock time to reach tau on the Marshak wave (FP64 path, the host
    driver setting the boundary from the Su & Olson quadrature before every subcycle, as the paper's
    code does), for each N and tau; the oracle timed the same way on the runs it finishes quickly."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import torch

    torch.cuda.set_device(0)
    from paper_1306_0010_gb300 import build, rhd, workloads as wl

    build.build()
    rhd.lib()
    Ns = tuple(int(v) for v in args.marshak_sizes.split(","))
    taus = tuple(float(v) for v in args.marshak_taus.split(","))
    # warm-up (first launches of both precisions' kernels, library set-up)
    for precision in ("fp64", "split"):
        w = wl.marshak_case(64, precision=precision)
        g = rhd.Grid(dict(w["desc"], flags=rhd.FLAG_NO_GRAPH))
        g.load_case(w)
        g.marshak_advance(20, w["chat"], w["dt"], 0.0, w["marshak"])
        g.synchronize()
        g.close()
    table = []
    for N in Ns:
        for tau in taus:
            case = wl.marshak_case(N)
            n_sub = wl.marshak_subcycles(tau, case)
            g = rhd.Grid(dict(case["desc"], flags=rhd.FLAG_NO_GRAPH))
            g.load_case(case)
            g.synchronize()
            t0 = time.perf_counter()
            g.marshak_advance(n_sub, case["chat"], case["dt"], 0.0, case["marshak"])
            g.synchronize()
            el = time.perf_counter() - t0
            g.close()
            row = {"N": N, "tau": tau, "n_sub": n_sub, "gpu_s": el, "gpu_cell_updates_per_s": N * n_sub / el,
                   "gpu_split_s": None, "cpu_s": None}
            # the same run on the split path (FP32 fluxes and closure, FP64 accumulation and exchange)
            cs = wl.marshak_case(N, precision="split")
            g = rhd.Grid(dict(cs["desc"], flags=rhd.FLAG_NO_GRAPH))
            g.load_case(cs)
            g.synchronize()
            t0 = time.perf_counter()
            g.marshak_advance(n_sub, cs["chat"], cs["dt"], 0.0, cs["marshak"])
            g.synchronize()
            row["gpu_split_s"] = time.perf_counter() - t0
            g.close()
            if N * n_sub <= args.marshak_cpu_cells:
                row["cpu_s"] = marshak_oracle_seconds(case, n_sub)
            table.append(row)
    # the kernels' own time per subcycle (events around each launch), against the wall clock per subcycle
    kernel_us = {}
    for precision in ("fp64", "split"):
        case = wl.marshak_case(max(Ns), precision=precision)
        n_sub = wl.marshak_subcycles(min(10.0, max(taus)), case)
        g = rhd.Grid(dict(case["desc"], flags=rhd.FLAG_NO_GRAPH))
        g.load_case(case)
        g.set_kernel_timing(True)
        g.marshak_advance(n_sub, case["chat"], case["dt"], 0.0, case["marshak"])
        g.synchronize()
        kt = g.kernel_times()
        g.close()
        kernel_us[precision] = {k: 1e3 * v["total_ms"] / v["launches"] for k, v in kt.items()}
    big = table[-1]
    line = {"metric": "non-equilibrium Marshak wave (Section 4.1.4): wall-clock time to reach tau", "value": big["gpu_s"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1D Marshak wave, chi in [0, 100], rho = kappa_0 = 1, eps = 1, a_R = c = chat = 1, "
                                   "F_inc = 1/4, linear exchange, theta = 1, CFL 0.4, boundary from the midpoint "
                                   "quadrature (1024 points) before every subcycle; value: the largest N at the largest tau",
                       "N": big["N"], "tau": big["tau"]},
            "table": table, f"kernel_us_per_subcycle_{max(Ns)}": kernel_us, "vs_baseline": None}
    print(json.dumps(line), flush=True)


def marshak_oracle_seconds(case, n_sub):
    """The oracle driven like the library: the boundary state before every subcycle, one subcycle per call."""
    import copy

    from oracle import marshak, oracle as orc

    c = copy.deepcopy(case)
    m = c["marshak"]
    t0 = time.perf_counter()
    for k in range(n_sub):
        tau = m["tau_rate"] * (k + 0.5) * c["dt"]
        E_b, F_b = marshak.boundary_state(tau, m["eps"], m["F_inc"], c["desc"]["c"], 1024)
        c["desc"]["dirichlet_lo"][0] = [E_b, F_b, 0.0, 0.0]
        st, _ = orc.subcycles(c, n_sub=1)
        c["fields"] = dict(c["fields"], E=st["E"], Fx=st["Fx"], Fy=st["Fy"], Fz=st["Fz"], T=st["T"])
    return time.perf_counter() - t0


def run_ensemble(args):
    import torch

    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(lrank)
    from paper_1306_0010_gb300 import build, rhd, workloads as wl

    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    rhd.lib()
    n_sub = args.ens_n_sub
    cases = wl.config5(n_grids=args.n_grids, n_sub=n_sub, precision="split")
    cells = sum(int(np.prod(c["desc"]["n"])) for c in cases)
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()
    res = {}
    clk = ClockSampler(lrank)
    clk.start()
    # the FP64 path is ~30x slower: fewer subcycles and steps keep the run within minutes
    plan = {"split": (n_sub, args.steps, args.warmup), "fp64": (max(1, n_sub // 5), 2, 1)}
    for prec in ("split", "fp64"):
        ns, steps, warm = plan[prec]
        ms, chosen, kt, st = time_ensemble(torch, rhd, cases, prec, ns, steps, warm, stream)
        base_ms = time_per_grid(torch, rhd, cases, prec, ns, steps, 1, stream)
        if ws > 1:
            ms = max_over_ranks(ms, dist, device="cuda")
            base_ms = max_over_ranks(base_ms, dist, device="cuda")
        res[prec] = {"value": whole_job_rate(cells, ns, steps, ws, ms), "ms_per_step": ms / steps,
                     "n_sub_per_step": ns, "steps": steps,
                     "per_grid_plain_launches": whole_job_rate(cells, ns, steps, ws, base_ms),
                     "launch": chosen, "roofline": kernel_roofline(kt, hbm_peak, peak_kind),
                     "stats": {k: st[k] for k in ("n_realizability_fix", "n_theta_fallback", "n_nonfinite",
                                                  "newton_iter_max")}}
        res[prec]["speedup_vs_per_grid"] = res[prec]["value"] / res[prec]["per_grid_plain_launches"]
    clocks = clk.stop()
    if rank == 0:
        sp = res["split"]
        line = {"metric": METRIC, "value": sp["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": sp["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
                "config": dict(ensemble_workload_config(args, cases), precision="split"),
                "roofline": sp["roofline"], "clocks": clocks,
                "gpu_launches": args.steps * n_sub, "split": sp, "fp64": res["fp64"]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.traffic_from:
        return record_traffic(args.traffic_from, args.N, 512, args.launch)
    if args.fp64_ops_from:
        return record_fp64_ops(args.fp64_ops_from, args.N)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "marshak":
        return run_marshak(args)
    import torch

    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(lrank)
    from paper_1306_0010_gb300 import build, rhd, workloads as wl

    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    rhd.lib()
    case = wl.config4(N=args.N, n_sub=args.n_sub)
    cells = args.N ** 3
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()

    # headline: split path; every rank advances its own independent grid (replicas, no exchange)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(lrank)
    clk.start()
    total_ms, per_step, st, kt, launch, tuning, rsla = time_path(torch, rhd, case, "split", args.n_sub, args.steps,
                                                                 args.warmup, stream, launch_spec=args.launch,
                                                                 rsla_peak=hbm_peak, peak_kind=peak_kind)
    clocks = clk.stop()
    if ws > 1:
        total_ms = max_over_ranks(total_ms, dist, device="cuda")
        dist.barrier()
    value = whole_job_rate(cells, args.n_sub, args.steps, ws, total_ms)
    sub_ms = total_ms / (args.steps * args.n_sub)
    roofline = kernel_roofline(kt, hbm_peak, peak_kind)
    # the dominant kernel (the corrector, which completes every cell-update) against the method's own
    # bytes per cell-update (B_alg of the split path: U^m read, U^{m+1} written, T read and written, the
    # FP32 gas read) times the cells of one launch; the kernel's own design bytes (with U^{m+1/2} and the
    # FP32 mirror the two-pass design adds) are reported beside it
    design = roofline["alg_bytes_per_launch"]
    roofline["alg_bytes_per_launch"] = float(B_ALG["split"] * cells)
    roofline["achieved"] = roofline["alg_bytes_per_launch"] / (roofline["launch_ms"] * 1e-3) / 1e9
    roofline["frac"] = roofline["achieved"] / hbm_peak
    roofline["bytes_per_cell_update"] = B_ALG["split"]
    roofline["design_bytes_per_launch"] = design
    roofline["design_frac"] = design / (roofline["launch_ms"] * 1e-3) / 1e9 / hbm_peak
    traffic_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_path):
        trj = json.load(open(traffic_path))
        tr = trj.get(roofline["kernel"])
        # the corrector's DRAM traffic does not depend on the z chunk (its only per-chunk extra is four
        # planes of one column): match variant, tile and staging
        def same_kernel(a, b):
            return a.split(":")[:2] + a.split(":")[3:] == b.split(":")[:2] + b.split(":")[3:]
        if (tr and tr.get("N") == args.N and same_kernel(tr.get("launch", ""), launch_key(launch))
                and trj.get("source_sha256") == kernel_source_hash()):
            roofline["traffic"] = tr["bytes_per_launch"]
            roofline["traffic_over_alg"] = tr["bytes_per_launch"] / roofline["alg_bytes_per_launch"]
            tp = trj.get("twopass_predictor_split")
            if tp and tp.get("N") == args.N:
                # the whole subcycle's DRAM traffic over the method's bytes (re-reads and the two-pass extras)
                roofline["subcycle_traffic_over_alg"] = (tr["bytes_per_launch"] + tp["bytes_per_launch"]) / (
                    B_ALG["split"] * cells)
    # the whole subcycle against the method's own bytes per cell-update (U^m, gas, T in; U^{m+1}, T out)
    sub_achieved = B_ALG["split"] * cells / (sub_ms * 1e-3) / 1e9
    subcycle_roofline = {"bound": "hbm", "achieved": sub_achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": sub_achieved / hbm_peak, "bytes_per_cell_update": B_ALG["split"],
                         "subcycle_ms": sub_ms}

    extra = {}
    if not args.no_fp64:
        fp_ms, fp_steps, fst, fkt, flaunch, _, _ = time_path(torch, rhd, case, "fp64", args.fp64_n_sub,
                                                             max(2, args.steps // 2), args.warmup, stream)
        fn = max(2, args.steps // 2)
        if ws > 1:
            fp_ms = max_over_ranks(fp_ms, dist, device="cuda")
        fv = whole_job_rate(cells, args.fp64_n_sub, fn, ws, fp_ms)
        f_launch = fp_ms / (fn * args.fp64_n_sub)
        extra["fp64_path"] = {"value": fv, "unit": UNIT, "n_sub_per_step": args.fp64_n_sub,
                              "launch_ms": f_launch, "split_speedup": value / fv, "launch": flaunch,
                              "roofline": kernel_roofline(fkt, hbm_peak, peak_kind),
                              "fp64_pipe_roofline": fp64_pipe_roofline(fv / ws)}
    e2e = None
    if not args.no_e2e and rank == 0:
        n_e = max(4, args.steps)
        el, h2d, d2h = time_e2e(torch, rhd, case, "split", args.n_sub, n_e, 1, args.launch)
        e2e = {"value": cells * args.n_sub * n_e / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e,
               "pipelining": "two grids on two streams take the steps in turn: one step's copies overlap "
                             "the other grid's subcycles"}
    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_baseline(case, args.cpu_seconds)
    configs = None
    if not args.no_configs and rank == 0:
        configs = {"config1_linear_wave": run_config1(torch, rhd, wl, stream),
                   "config2_source_2d": run_config2(torch, rhd, wl, stream),
                   "config3_shell": run_config3(torch, rhd, wl, stream, hbm_peak),
                   "config5_ensemble": run_config5(torch, rhd, wl, stream, hbm_peak, peak_kind),
                   "config4_far_from_equilibrium": run_far_from_equilibrium(torch, rhd, case, launch, stream,
                                                                            roofline.get("launch_ms"))}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
                "config": dict(workload_config(args, "split"), launch=launch),
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": sum(v["launches"] for v in kt.values()), "clocks": clocks,
                "subcycle_roofline": subcycle_roofline, "alu_roofline": alu_roofline(value / ws),
                "kernels": kt, "autotune": tuning, "rsla": rsla,
                "gas_step": rsla.pop("gas_step", None) if rsla else None,
                "stats": {k: st[k] for k in ("n_realizability_fix", "n_face_fallback", "n_theta_fallback",
                                             "n_nonfinite", "newton_iter_max")},
                "per_step_ms": per_step, "configs": configs}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
