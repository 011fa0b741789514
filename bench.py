"""Benchmark: DOF-updates/s of the blended RHS + SSP-RK3 stage on one GB300.

Workload (default): 2D Sedov blast, M = 8 mean values per direction per element
(the paper's N = 8: hierarchy FV, 2x2, 4x4 sub-elements and full order), 256^2
elements on [-1,1]^2 with reflecting walls, gamma = 1.4, CFL 0.5; measured in the
FP32-split form (the headline) and in plain FP64 (reported beside it). One step
is one SSP-RK3 step through the C ABI: the time-step reduction and three stages,
each stage the indicator kernel, the interface-flux kernel and the update kernel.
DOF = one subcell mean value with all conserved variables; every stage updates
E * M^d of them.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun) every rank advances its own independent replica of the
workload (no data-path collective); the step time is the maximum over ranks and
`value` counts the DOF updates of all ranks.
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
# the CPU oracle legs are timed on one host thread (their reported `cores`): keep
# numpy's BLAS single-threaded (the GPU legs do no BLAS work on the host)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "DOF-updates/s of blended RHS+RK stage (FP64 vs FP32-split) and % HBM roofline"
UNIT = "DOF-updates/s"
WORKLOAD = "sedov2d_M8_256x256"
RK_STAGES = 3
FP64_PEAK_UNITS = (152, 2, 2070.0)    # SMs, FP64 FMA per clock per SM, max SM clock (MHz)
FP32_PEAK_UNITS = (152, 128, 2070.0)  # SMs, FP32 FMA per clock per SM, max SM clock (MHz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sesc", choices=["sesc", "reference"])
    ap.add_argument("--nel", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched ensemble (profiling runs) and print its object")
    ap.add_argument("--precisions", default="fp32_split,fp64",
                    help="comma list; the first is the headline (profiling runs may pick one)")
    return ap.parse_args()


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _smi_id(index):
    """nvidia-smi id of CUDA device `index` of this process (CUDA_VISIBLE_DEVICES
    renumbers devices; its entries are indices or UUIDs, both accepted by --id)."""
    vis = [x.strip() for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    return vis[index] if index < len(vis) else str(index)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background;
    mark() brackets the timed region, and the summary keeps the samples taken
    inside it (all samples, flagged, when none falls inside)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.marks = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={_smi_id(self.index)}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def mark(self):
        """Wall-clock time (local, as nvidia-smi prints it) at a bracket of the timed region."""
        import datetime
        self.marks.append(datetime.datetime.now())

    def summary(self):
        self.f.flush()
        with open(self.f.name) as fh:
            text = fh.read()
        os.unlink(self.f.name)
        return self.parse(text, self.marks)

    @classmethod
    def parse(cls, text, marks=()):
        import datetime
        rows = []
        for line in text.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                ts = None
            rows.append((ts, parts[1:]))
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0, "samples_in_region": 0}
        inside = rows
        if len(marks) >= 2:
            inside = [r for r in rows if r[0] is not None and marks[0] <= r[0] <= marks[-1]]
        use = inside if inside else rows

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1][1]) for r in use) if v is not None]
        smax = [v for v in (num(r[1][2]) for r in use) if v is not None]
        pw = [v for v in (num(r[1][3]) for r in use) if v is not None]
        reasons = sorted({cls.NAMES[i] for r in use for i in range(4) if r[1][5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(use), "samples_in_region": len(inside) if len(marks) >= 2 else None,
                "power_w_max": max(pw) if pw else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def flops_update_pure_top(M, d):
    """Algorithmic FP64 flops of the update kernel for one element whose only
    active level is the top one (the dominant element class): reconstruction
    (d passes of an M-point contraction per mean and variable), nodal fluxes,
    volume operator (d passes per direction), surface columns, blend and RK.
    An FMA counts 2, a divide 1."""
    nv, MD = d + 2, M ** d
    recon = d * nv * MD * 2 * M
    flux = d * MD * 12
    volume = d * d * nv * MD * 2 * M
    surface = d * nv * MD * 5
    blend_rk = nv * MD * 6
    return recon + flux + volume + surface + blend_rk


def _oracle_window(cfg, u, window):
    """The central window x window elements of the state as an oracle problem (walls
    around the window): (grid state, oracle Config, window side)."""
    from oracle.blended import Config
    from oracle.layout import to_grid
    M, n = cfg["M"], cfg["nel"][0]
    w = min(window, n)
    lo = (n - w) // 2
    U = to_grid(u, 2, M, cfg["nel"])[:, lo * M:(lo + w) * M, lo * M:(lo + w) * M].copy()
    dx = (cfg["xhi"][0] - cfg["xlo"][0]) / n
    sub = dict(cfg)
    sub.update(nel=(w, w), xlo=(cfg["xlo"][0] + lo * dx,) * 2, xhi=(cfg["xlo"][0] + (lo + w) * dx,) * 2)
    return U, Config(**sub), w


def oracle_sample_rate(cfg, u, seconds=12.0, window=48):
    """The CPU oracle, as it stands, on a bounded sample of the workload: the
    central window x window elements of the state, each step one SSP-RK3 step of
    the oracle on that window (walls around it). Returns (DOF-updates/s, sample
    description, steps run, threads)."""
    from oracle.timestep import rk3_step
    U, c, w = _oracle_window(cfg, u, window)
    M, n = cfg["M"], cfg["nel"][0]
    t0 = time.perf_counter()
    steps = 0
    while True:
        U, _ = rk3_step(U, c)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    dof = w * w * M ** 2 * RK_STAGES * steps
    desc = (f"oracle (numpy FP64) SSP-RK3 steps on the central {w}x{w} elements (M={M}) of the "
            f"{n}x{n} Sedov state, walls around the window; {steps} steps in {el:.1f} s")
    return dof / el, desc, steps, 1


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, as it stands, timed on the host cores on the
    same workload and metric: W untimed and K timed oracle SSP-RK3 steps, each on the
    central window of the Sedov state, the window sized so that the W + K steps take
    about two minutes at most (48 x 48 elements, about 2.7 s per step on one x86 core,
    for K + W <= 44)."""
    from oracle.timestep import rk3_step
    from paper_2011_03338_gb300 import inputs
    if rank != 0:
        return
    cfg, u = inputs.sedov(2, 8, args.nel)
    n_steps = max(1, args.warmup + args.steps)
    window = max(8, min(48, int(48 * math.sqrt(44.0 / n_steps))))
    U, c, w = _oracle_window(cfg, u, window)
    M, n = cfg["M"], cfg["nel"][0]
    for _ in range(args.warmup):
        U, _ = rk3_step(U, c)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _ = rk3_step(U, c)
    el = time.perf_counter() - t0
    rate = w * w * M ** 2 * RK_STAGES * args.steps / max(el, 1e-9)
    desc = (f"oracle (numpy FP64) SSP-RK3 steps on the central {w}x{w} elements (M={M}) of the "
            f"{n}x{n} Sedov state, walls around the window; {args.warmup} untimed + {args.steps} timed "
            f"steps, {el:.1f} s timed")
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(cfg, u, precision, args, world):
    """Warm-up, then K timed SSP-RK3 steps of one precision; per-kernel CUDA-event
    times recorded by the library inside the timed region; clocks sampled."""
    import torch
    from paper_2011_03338_gb300 import Solver
    s = Solver(dict(cfg, precision=precision))
    stream = torch.cuda.current_stream()
    ua = torch.from_numpy(u).cuda()
    ub = torch.empty_like(ua)
    dt_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        s.rk3_step(ua, ub, dt_dev)
        ua, ub = ub, ua
    torch.cuda.synchronize()
    rc, _ = s.status()
    if rc != 0:
        raise RuntimeError(f"device status after warm-up ({precision}): {rc}")
    s.set_timing(True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk.mark()
        e0.record(stream)
        for _ in range(args.steps):
            s.rk3_step(ua, ub, dt_dev)
            ua, ub = ub, ua
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark()
        barrier(world)
    ms = e0.elapsed_time(e1)
    times = s.kernel_times()
    s.set_timing(False)
    rc, counters = s.status()
    if rc != 0:
        raise RuntimeError(f"device status after timed steps ({precision}): {rc}")
    return s, max_over_ranks(ms, world), times, clk.summary(), counters, dt_dev


def e2e_run(s, u, args, world, dt_dev):
    """The same steps through the public API (Solver.rk3_step), with every step's state
    copied in from pinned host memory and its result copied back to pinned host
    memory. The copies run on their own streams with double-buffered device and host
    buffers, so the copy-in for step k+1 and the copy-out of step k-1 overlap the
    kernels of step k, as a caller streaming states through the library would do."""
    import torch
    main = torch.cuda.current_stream()
    cs, si, so = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    uh = torch.from_numpy(u).pin_memory()
    oh = [torch.empty_like(uh).pin_memory() for _ in range(2)]
    din = [torch.empty(uh.shape, dtype=uh.dtype, device="cuda") for _ in range(2)]
    dout = [torch.empty_like(din[0]) for _ in range(2)]
    in_ready, in_free, done, out_free = ([torch.cuda.Event() for _ in range(2)] for _ in range(4))

    def run(steps):
        for e in in_free + out_free:
            e.record(main)
        for k in range(steps):
            i = k % 2
            si.wait_event(in_free[i])
            with torch.cuda.stream(si):
                din[i].copy_(uh, non_blocking=True)
            in_ready[i].record(si)
            cs.wait_event(in_ready[i])
            cs.wait_event(out_free[i])
            with torch.cuda.stream(cs):
                s.rk3_step(din[i], dout[i], dt_dev)
            done[i].record(cs)
            in_free[i].record(cs)
            so.wait_event(done[i])
            with torch.cuda.stream(so):
                oh[i].copy_(dout[i], non_blocking=True)
            out_free[i].record(so)
        for st in (si, cs, so):
            main.wait_stream(st)

    for st in (si, cs, so):
        st.wait_stream(main)
    run(2)
    torch.cuda.synchronize()
    barrier(world)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(main)
    for st in (si, cs, so):
        st.wait_stream(main)
    run(args.steps)
    f1.record(main)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(f0.elapsed_time(f1), world), uh.numel() * 8


def kernel_sources_sha256(precision):
    """Hash of the sources the kernels of one precision are compiled from."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2011_03338_gb300", "csrc")
    files = ["blend_kernels.cuh", "kparams.h", "kernels_fp64.cu" if precision == "fp64" else "kernels_split.cu"]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel, precision, nel):
    """DRAM bytes per launch of `kernel` from the ncu summary under profiles/, or
    None when there is none for this workload or the kernel sources changed since."""
    if nel != 256:
        return None, "no ncu capture of this workload"
    tag = "split" if precision == "fp32_split" else "fp64"
    path = os.path.join(ROOT, "profiles", f"{kernel}_{tag}_sedov2d_M8_256.md")
    if not os.path.exists(path):
        return None, "no ncu capture"
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.split(":")[0] in ("traffic_bytes_per_launch", "sources_sha256"):
                k, v = line.split(":", 1)
                fields[k] = v.strip()
    if fields.get("sources_sha256") != kernel_sources_sha256(precision):
        return None, "kernel changed since the ncu capture"
    return int(fields["traffic_bytes_per_launch"]), os.path.relpath(path, ROOT)


def roofline_of(times, E, M, d, ms_per_step, peaks, peak_src, fp64, nel=256):
    avg_ms = {k: (times[k][0] / times[k][1] if times[k][1] else None) for k in times}
    total = max(1e-9, sum(v[0] for v in times.values()))
    dominant = max(("indicator", "face_flux", "update"), key=lambda k: times[k][0])
    if fp64:
        peak = FP64_PEAK_UNITS[0] * FP64_PEAK_UNITS[1] * 2 * FP64_PEAK_UNITS[2] * 1e6 / 1e12
        src = ("derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz (FP64 is not in MEASURED_PEAKS.json; "
               "a probe measured 1.19 TFLOP/s at 1995 MHz)")
    else:
        peak = FP32_PEAK_UNITS[0] * FP32_PEAK_UNITS[1] * 2 * FP32_PEAK_UNITS[2] * 1e6 / 1e12
        src = ("derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz (a probe measured 69.5 TFLOP/s "
               "at 1995 MHz)")
    upd_flops = flops_update_pure_top(M, d) * E
    achieved = upd_flops / (avg_ms["update"] * 1e-3) / 1e12
    state_bytes = E * (d + 2) * M ** d * 8
    hbm_bytes_stage = 3 * state_bytes
    stage_ms = ms_per_step / RK_STAGES
    traffic, traffic_src = profiled_traffic("k_update", "fp64" if fp64 else "fp32_split", nel)
    return {"bound": "alu", "kernel": "k_update (level RHS in subcell-flux form, blend, RK stage)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_source": traffic_src,
            "peak_source": src, "flops_per_launch": upd_flops,
            "kernel_ms": avg_ms, "kernel_share": {k: times[k][0] / total for k in times},
            "dominant_by_time": dominant,
            "hbm": {"algorithmic_bytes_per_stage": hbm_bytes_stage,
                    "achieved_gbs": hbm_bytes_stage / (stage_ms * 1e-3) / 1e9,
                    "peak_gbs": peaks["hbm_gbs"], "peak_source": peak_src,
                    "frac": hbm_bytes_stage / (stage_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}}


def adjoint_cost(args):
    """FP64 stage adjoint (sesc_rk_stage_vjp, frozen coefficients) against the FP64
    forward stage (sesc_rk_stage) on the Kelvin-Helmholtz adjoint workload: periodic
    [-1,1]^2, M = 8, 128^2 elements; CUDA events, best of a few repetitions."""
    import torch
    from paper_2011_03338_gb300 import Solver, inputs
    cfg, u = inputs.kelvin_helmholtz(8, 128, seed=0)
    s = Solver(dict(cfg, precision="fp64"))
    us = torch.from_numpy(u).cuda()
    out = torch.empty_like(us)
    c = torch.empty((s.E, 2, s.S), dtype=torch.float64, device="cuda")
    g = torch.ones_like(us)
    us_bar = torch.empty_like(us)
    u0_bar = torch.zeros_like(us)
    dt = 1e-4

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    fwd = timed(lambda: s.rk_stage(us, us, out, 0.75, 0.25, dt=dt, coeffs_out=c), 5)
    adj = timed(lambda: s.rk_stage_vjp(us, g, us_bar, 0.75, 0.25, dt=dt, frozen=c, u0_bar=u0_bar), 5)
    s.close()
    return {"workload": "kelvin_helmholtz M=8 128x128 elements, FP64, one RK stage", "forward_ms": fwd,
            "adjoint_ms": adj, "adjoint_over_forward": adj / fwd}


def batched_ensemble(args):
    """The batched workload: 64 independent four-quadrant problems (seeded states,
    meshes 32^2 .. 256^2 elements, M in {4, 8}, FP32-split, outflow), one SSP-RK3
    step of every problem per step with its own time step. Timed three ways with
    CUDA events after warm-up: the batch replaying its captured CUDA graph at
    autotuned grids (the configuration reported as `value`), the same batch
    launched eagerly, and one standalone handle per problem stepped in a loop."""
    import torch
    from paper_2011_03338_gb300 import Batch, Solver, inputs
    probs = inputs.quadrant_ensemble(64, seed=0, precision="fp32_split")
    dof_step = sum(int(c["nel"][0] * c["nel"][1]) * c["M"] ** 2 for c, _ in probs) * RK_STAGES
    b = Batch([c for c, _ in probs])
    ua = torch.empty(b.total, dtype=torch.float64, device="cuda")
    for k, (_, uk) in enumerate(probs):
        b.view(ua, k).copy_(torch.from_numpy(uk))
    u0 = ua.clone()
    ub = torch.empty_like(ua)
    dt = torch.empty(len(probs), dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    grids = b.autotune(ua, reps=3)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def timed(step, steps):
        nonlocal ua, ub
        for _ in range(args.warmup):
            step(ua, ub)
            ua, ub = ub, ua
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(ua, ub)
            ua, ub = ub, ua
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    b.use_graph(True)
    ms_graph = timed(lambda x, y: b.rk3_step(x, y, dt), args.steps)
    b.use_graph(False)
    ua.copy_(u0)
    ms_eager = timed(lambda x, y: b.rk3_step(x, y, dt), args.steps)
    rc, cs = b.status()
    flagged = sum(1 for c in cs if c[0] & 1)
    bad_final = sum(1 for c in cs if c[0] & 2)
    groups = [{"M": probs[b.group_of.index(g)][0]["M"], "problems": b.group_of.count(g),
               "grids": dict(zip(("indicator", "face_flux", "update", "dt"), grids[g]))} for g in range(b.ngroups)]
    total = b.total
    b.close()
    # one handle per problem, stepped one after the other
    solvers, states = [], []
    for c, uk in probs:
        solvers.append(Solver(c))
        x = torch.from_numpy(uk).cuda()
        states.append([x, torch.empty_like(x)])
    dt1 = torch.empty(1, dtype=torch.float64, device="cuda")

    def loop_step(_x, _y):
        for s, st in zip(solvers, states):
            s.rk3_step(st[0], st[1], dt1)
            st.reverse()
    ms_loop = timed(loop_step, max(2, args.steps // 2))
    for s in solvers:
        s.close()
    ngroups = len(groups)
    return {"workload": "quadrants_ensemble_64 (2D four-quadrant Riemann problems, 32^2..256^2 elements, "
                        "M in {4,8}, FP32-split)",
            "problems": len(probs), "elements": sum(int(c["nel"][0] * c["nel"][1]) for c, _ in probs),
            "state_bytes": total * 8, "value": dof_step / (ms_graph * 1e-3), "unit": UNIT,
            "ms_per_step": ms_graph, "eager_ms_per_step": ms_eager, "per_problem_loop_ms_per_step": ms_loop,
            "speedup_over_per_problem_loop": ms_loop / ms_graph,
            "kernel_launches_per_step": ngroups * (2 + RK_STAGES * 3),
            "autotune_s": tune_s, "groups": groups,
            "problems_with_nonpermissible_stage": flagged, "problems_with_nonfinite_dt": bad_final}


def sedov3d(args):
    """The 3D workload: Sedov blast on [-1,1]^3, M = 8 (512 means per element), 64^3
    elements, walls; one warm-up and two timed SSP-RK3 steps per precision (CUDA
    events), per-kernel times from the library."""
    import torch
    from paper_2011_03338_gb300 import Solver, inputs
    nel = 64
    cfg, u = inputs.sedov(3, 8, nel)
    dof_step = nel ** 3 * 512 * RK_STAGES
    out = {"workload": "sedov3d_M8_64x64x64", "elements": nel ** 3, "steps": 2}
    for prec in ("fp32_split", "fp64"):
        s = Solver(dict(cfg, precision=prec))
        a = torch.from_numpy(u).cuda()
        b = torch.empty_like(a)
        dt = torch.empty(1, dtype=torch.float64, device="cuda")
        s.rk3_step(a, b, dt)
        a, b = b, a
        torch.cuda.synchronize()
        s.set_timing(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            s.rk3_step(a, b, dt)
            a, b = b, a
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        kt = s.kernel_times()
        rc, _ = s.status()
        out[prec] = {"value": dof_step / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "status": rc,
                     "kernel_ms": {k: (v[0] / v[1] if v[1] else None) for k, v in kt.items()}}
        s.close()
        del a, b
        torch.cuda.empty_cache()
    out["split_speedup_over_fp64"] = out["fp32_split"]["value"] / out["fp64"]["value"]
    return out


def main():
    args = parse()
    rank, world = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    from paper_2011_03338_gb300 import inputs
    if args.only_batched:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "batched": batched_ensemble(args), "note": "partial run"}), flush=True)
        return

    cfg, u = inputs.sedov(2, 8, args.nel)
    M, d = cfg["M"], cfg["dim"]
    E = cfg["nel"][0] * cfg["nel"][1]
    dof_per_step = E * M ** d * RK_STAGES
    peaks, peak_src = measured_peaks()
    launches_per_step = 3 + RK_STAGES * (1 + d + 1)   # two wave-speed passes + dt, then K1, K2 per direction, K3

    results = {}
    precs = [x for x in args.precisions.split(",") if x]
    for prec in precs:
        s, ms, times, clocks, counters, dt_dev = measure(cfg, u, prec, args, world)
        ms_per_step = ms / args.steps
        res = {"value": dof_per_step * args.steps * world / (ms * 1e-3), "ms_per_step": ms_per_step,
               "roofline": roofline_of(times, E, M, d, ms_per_step, peaks, peak_src, prec == "fp64", args.nel),
               "clocks": clocks,
               "counters": {"squeezed": counters[1], "dropped_dg_blocks": counters[2],
                            "n_min_hist": counters[4:8], "n_max_hist": counters[8:12]}}
        if prec == "fp32_split" and not args.no_e2e:
            ems, nbytes = e2e_run(s, u, args, world, dt_dev)
            res["e2e"] = {"value": dof_per_step * args.steps * world / (ems * 1e-3), "unit": UNIT,
                          "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                          "ms_per_step": ems / args.steps,
                          "input": "the workload's initial state, copied in every step (the device-timed "
                                   "loop advances the blast instead)"}
        s.close()
        results[prec] = res

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, desc, steps, cores = oracle_sample_rate(cfg, u)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0 and len(precs) == 1:
        r = results[precs[0]]
        print(json.dumps({"metric": METRIC, "value": r["value"], "unit": UNIT, "precision": precs[0],
                          "ms_per_step": r["ms_per_step"], "roofline": r["roofline"], "note": "partial run"}))
    elif rank == 0:
        head = results["fp32_split"]
        fp64 = results["fp64"]
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 split", "data": "synthetic",
                "config": {"workload": WORKLOAD, "dim": d, "M": M, "elements": E, "dof": E * M ** d,
                           "precision": "fp32_split (headline); fp64 beside it",
                           "step": "dt + 3 SSP-RK3 stages (K1, K2 per direction, K3 each)",
                           "l2": "inputs larger than L2 (134 MB state, ~0.7 GB touched per stage)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head.get("e2e"),
                "clocks": head["clocks"], "counters": head["counters"],
                "fp64": {"value": fp64["value"], "unit": UNIT, "dtype": "f64", "ms_per_step": fp64["ms_per_step"],
                         "roofline": fp64["roofline"], "clocks": fp64["clocks"], "counters": fp64["counters"]},
                "split_speedup_over_fp64": head["value"] / fp64["value"],
                "adjoint": None if args.no_adjoint else adjoint_cost(args),
                "batched": None if args.no_batched else batched_ensemble(args),
                "sedov3d": None if args.no_3d else sedov3d(args)}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
