"""Benchmark: zone-updates/s of full ADER-WENO steps on one GB300 (or N
independent replicas under torchrun), with the ALU roofline of the dominant
kernel, clocks during the timed region, an end-to-end number through the C
ABI with host buffers, and the FP64 oracle timed on the host cores.

Workload (headline): 3D Euler, Taylor-Green vortex on a periodic 256^3 grid,
fourth-order WENO+ADER, HLLC, FP64, CFL 0.3 (device-resident dt).  One "step"
is one full step of the method over the whole grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# ALU peaks from unit counts and the maximum SM clock: 152 SMs x 2 FP64 FMA
# lanes/clk (x 128 FP32) x 2 flops x 2.07 GHz
SMS, CLK = 152, 2.07e9
PEAK_FP64 = SMS * 2 * 2 * CLK / 1e12      # 1.259 TFLOP/s
PEAK_FP32 = SMS * 128 * 2 * CLK / 1e12    # 80.5 TFLOP/s


def hbm_peak():
    """measured copy bandwidth of the GB300s (GB/s), else the
    profiling recipe's fallback"""
    try:
        return float(json.load(open(MEASURED_PEAKS))["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--order", type=int, default=4, choices=[2, 3, 4],
                    help="order of the TGV workload (4: the headline; 2, 3 for profiling)")
    ap.add_argument("--form", default="fp64", choices=["fp64", "fp32"],
                    help="arithmetic form of the headline line (fp64 is the workload's)")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32-bulk form line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--gate", action="store_true",
                    help="time the headline grid with the gate on (He-initialised weights; for profiling)")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "native":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return rank, world, local


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


# --------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region"""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out["sm_mhz"] = float(np.median(sm)) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


# --------------------------------------------------------------------------
def workload(n, order=4):
    from paper_2211_13295_gb300 import problems as P
    return P.tgv3d(n=n, order=order, cfl=0.3)


def workload_name(prob):
    ext = f"{prob.n[0]}^3" if prob.n[2] == prob.n[0] else f"{prob.n[0]}x{prob.n[1]}x{prob.n[2]}"
    return f"tgv3d {ext} order {prob.order} HLLC CFL {prob.cfl} periodic"


def gpu_state(prob):
    """initial state generated on the host (exact zone averages), as a pinned tensor"""
    import torch
    U = prob.initial_state()
    return torch.from_numpy(U).pin_memory()


def time_steps(grid, steps, warmup, world):
    import torch
    grid.cfl_dt()
    for _ in range(warmup):
        grid.step(0.0, sync=False)
    grid.check()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    grid.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        grid.step(0.0, sync=False)
    e1.record()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = grid.profile_read()
    grid.profile(False)
    grid.check()
    return ms, prof


def time_e2e(grid, Uh, steps, world):
    """through the public API with host buffers: H2D of the state from pinned
    memory, one step, D2H of the updated state, every step"""
    import torch
    out = torch.empty_like(Uh).pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        grid.set_state(Uh.numpy())
        grid.step(0.0, sync=False)
        grid.get_state(out.numpy())
    torch.cuda.synchronize()
    barrier(world)
    return (time.perf_counter() - t0) * 1e3


def cpu_model():
    """the host CPU's model name (lscpu), else the architecture"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_one_core(order):
    """The oracle on one host core (OpenMP limited to one thread in a child
    process): one step of a periodic 16^3 Taylor-Green grid."""
    code = ("import sys, time; sys.path.insert(0, %r); import oracle; "
            "from paper_2211_13295_gb300 import problems as P; "
            "p = P.tgv3d(n=16, order=%d, cfl=0.3); U = p.initial_state(); o = oracle.Oracle(p); "
            "dt = o.cfl_dt(U, p.cfl); t0 = time.perf_counter(); o.step(U, 0.0, dt); "
            "print(p.zones / (time.perf_counter() - t0))") % (ROOT, order)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        v = float(out.stdout.strip().splitlines()[-1])
    except Exception as e:
        return {"value": None, "error": str(e)[:200]}
    return {"value": v, "unit": "zone-updates/s", "cores": 1,
            "sample": f"one step of tgv3d 16^3 order {order} FP64 (4096 zones), OMP_NUM_THREADS=1"}


def cpu_baseline_and_parity(prob, grid_state_after, U0, dt0, n_windows=3, m=4, seed=0):
    """The FP64 oracle (a) timed on a bounded sample of the workload (a full
    periodic 32^3 Taylor-Green grid, one step, all host cores) and (b) run on
    windows of the full-size grid to state the L1 error of the GPU step."""
    import oracle
    from paper_2211_13295_gb300 import problems as P
    cores = os.cpu_count()
    small = P.tgv3d(n=32, order=prob.order, cfl=prob.cfl)
    Us = small.initial_state()
    orc = oracle.Oracle(small)
    dts = orc.cfl_dt(Us, small.cfl)
    t0 = time.perf_counter()
    orc.step(Us, 0.0, dts)
    el = time.perf_counter() - t0
    base = {"value": small.zones / el, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"one step of tgv3d 32^3 order {prob.order} FP64 (32768 zones), {el:.1f} s wall",
            "cpu_model": cpu_model(), "one_core": oracle_one_core(prob.order)}
    # parity on windows of the full-size first step
    parity = None
    if grid_state_after is not None:
        g = prob.order
        rng = np.random.default_rng(seed)
        n = prob.n[0]
        L = prob.hi[0] - prob.lo[0]
        errs = []
        for _ in range(n_windows):
            c = rng.integers(0, n, size=3)
            idx = [np.arange(c[d] - g, c[d] + m + g) % n for d in range(3)]
            Ug = U0[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
            wprob = P.Problem("uniform", 3, (m, m, m), (0, 0, 0), (m * L / n,) * 3, prob.order,
                              cfl=prob.cfl)
            wo = oracle.Oracle(wprob)
            Uo, _, rc = wo.step_ghosted(Ug, dt0)
            sl = [np.arange(c[d], c[d] + m) % n for d in range(3)]
            Ugpu = grid_state_after[:, sl[2]][:, :, sl[1]][:, :, :, sl[0]]
            # relative L1 per variable, normalised by max(sum|U_v|, sum|rho|)
            # (rho*w of the Taylor-Green vortex starts at zero)
            sc = np.abs(Uo[0]).sum()
            e = max(np.abs(Ugpu[v] - Uo[v]).sum() / max(np.abs(Uo[v]).sum(), sc) for v in range(5))
            errs.append(e)
        parity = max(errs)
    return base, parity


def orders_192(args, world, scheme="ader", riemann="hllc", orders=(2, 3, 4), gate=None):
    """Zone-updates/s of the FP64 form at orders 2, 3 and 4 on a 192^3
    Taylor-Green grid: the grid of the paper's Tables II and IV (whose A100
    numbers were measured on an unnamed problem; context only).  scheme
    "ssprk" is Table IV's Runge-Kutta comparison (2, 3, 5 stages)."""
    from paper_2211_13295_gb300 import awe
    from paper_2211_13295_gb300 import problems as P
    out = {}
    for order in orders:
        prob = P.tgv3d(n=192, order=order, cfl=0.3).replace(scheme=scheme, riemann=riemann)
        g = awe.Grid(prob, gate=gate is not None)
        if gate is not None:
            g.gate_set_weights(gate)
        g.set_state(prob.initial_state())
        ms, prof = time_steps(g, 3, 3, world)
        ms = max_over_ranks(ms, world)
        g.close()
        out[f"O{order}"] = world * prob.zones * 3 / (ms * 1e-3)
        if len(orders) > 1:
            out[f"O{order}_stage_ms_per_step"] = {k: round(v[1] / 3, 3) for k, v in prof.items() if v[0]}
    return out


def other_configs(world, gate_params):
    """Zone-updates/s of the other workloads at their full sizes, in their
    forms: the double Mach reflection (4096x1024, order 3, FP32 bulk, with the
    positivity fallback), the Kelvin-Helmholtz layer (512^3, order 4, FP32
    bulk with the trained gate, 64-plane slabs) and the blast (384^3, order 4,
    FP64 with the trained gate and the a posteriori positivity fallback,
    128-plane slabs).  Two timed steps after one warm-up step each; the status
    after the timed steps is reported, and a run that ends non-physical has no
    rate."""
    import torch
    from paper_2211_13295_gb300 import awe
    from paper_2211_13295_gb300 import problems as P
    runs = [("dmr_4096x1024_o3_fp32_fallback", P.dmr(nx=4096, ny=1024).replace(fallback=True), "fp32", False, 0),
            ("kh3d_512_o4_fp32_gate_slab64", P.kh3d(n=512, order=4), "fp32", True, 64),
            ("blast3d_384_o4_fp64_gate_fallback2_slab128", P.blast3d(n=384, order=4).replace(fallback=2),
             "fp64", True, 128)]
    out = {}
    for name, prob, prec, gate, slab in runs:
        g = awe.Grid(prob, prec=prec, gate=gate, slab=slab)
        if gate:
            g.gate_set_weights(gate_params)
        g.set_state(prob.initial_state())
        g.cfl_dt()
        g.step(0.0, sync=False)
        torch.cuda.synchronize()
        g.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            g.step(0.0, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world) / 2
        prof = g.profile_read()
        g.profile(False)
        status = "ok"
        try:
            g.check()
        except awe.AweError as e:
            status = f"status {e.code}: {e}"
        # a run that ended in a non-physical state has no rate, only its status
        d = {"value": world * prob.zones / (ms * 1e-3) if status == "ok" else None, "unit": "zone-updates/s",
             "ms_per_step": ms if status == "ok" else None, "zones": prob.zones, "status": status,
             "stage_ms_per_step": {k: v[1] / 2 for k, v in prof.items() if v[0]}}
        if gate:
            fl, tot = g.gate_stats()
            d["flagged_fraction"] = fl / tot
        g.close()
        out[name] = d
    return out


def small_grid_graph():
    """The 2D workload (isentropic vortex, 64^2, order 3, CFL 0.4): a grid
    small enough that kernel launches dominate a step.  Per-step time of 100
    steps launched one by one, and of the same 100 steps replayed from one
    CUDA graph (awe.StepGraph), CUDA events on the grid's stream."""
    import torch
    from paper_2211_13295_gb300 import awe
    from paper_2211_13295_gb300 import problems as P
    prob = P.vortex2d(n=64, order=3)
    K = 100
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = awe.Grid(prob)
        g.set_state(prob.initial_state())
        g.cfl_dt()
        g.step(0.0, sync=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(K):
            g.step(0.0, sync=False)
        e1.record(s)
        s.synchronize()
        eager = e0.elapsed_time(e1) / K
        sg = awe.StepGraph(g, K, s)
        sg.replay()
        s.synchronize()
        e0.record(s)
        sg.replay()
        e1.record(s)
        s.synchronize()
        graph = e0.elapsed_time(e1) / K
        g.check()
        g.close()
    return {"workload": "vortex2d 64^2 order 3 HLLC CFL 0.4", "eager_ms_per_step": eager,
            "graph_ms_per_step": graph, "graph_zone_updates_per_s": prob.zones / (graph * 1e-3),
            "eager_zone_updates_per_s": prob.zones / (eager * 1e-3)}


def gated_forms(args, prob, Uh, U1, zones, world):
    """Train the troubled-zone gate on the GPU (labels from the method on
    short seeded runs of the vortex, Sod, blast and Kelvin-Helmholtz
    problems), then time the gated FP64 and FP32 forms on the same workload."""
    import torch
    from paper_2211_13295_gb300 import awe, gate_train
    from paper_2211_13295_gb300 import problems as P
    t0 = time.perf_counter()
    probs = [P.blast3d(n=48, order=4).replace(fallback=True), P.kh3d(n=48, order=4),
             P.tgv3d(n=48, order=4, cfl=0.3)]
    X, Y = gate_train.collect(probs, steps=(0, 3, 8))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    nin = X.shape[1]
    params, loss = gate_train.train(X, Y, nin, steps=1500, batch=8192)
    acc, recall, frac = gate_train.accuracy(params, X, Y, nin)
    t2 = time.perf_counter()
    collect_s, train_s = t1 - t0, t2 - t1
    out = {}
    for prec in ("fp64", "fp32"):
        g = awe.Grid(prob, prec=prec, gate=True)
        g.gate_set_weights(params)
        g.set_state(Uh.numpy())
        dt = g.cfl_dt()
        g.step(dt)
        fl, tot = g.gate_stats()
        Ug1 = g.get_state() if U1 is not None else None
        g.set_state(Uh.numpy())
        ms, prof = time_steps(g, args.steps, args.warmup, world)
        ms = max_over_ranks(ms, world)
        g.close()
        d = {"value": world * zones * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
             "flagged_fraction": fl / tot, "gate_ms_per_step": prof["gate"][1] / args.steps,
             "stage_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in prof.items() if v[0]}}
        if Ug1 is not None:
            sc = np.abs(U1[0]).sum()
            d["rel_l1_vs_full_weno_fp64_one_step"] = max(
                float(np.abs(Ug1[v] - U1[v]).sum() / max(np.abs(U1[v]).sum(), sc)) for v in range(5))
        out[f"{prec}_gated"] = d
    out["_params"] = params
    out["gate_training"] = {"rows": int(X.shape[0]), "positive_fraction": float(Y.mean()),
                            "accuracy": acc, "recall": recall, "train_seconds": train_s,
                            "collect_seconds": collect_s,
                            "final_loss": float(loss[-50:].mean())}
    return out


def slab_decomposition_1gpu(prob, Uh, U1, parts=2, steps=3, warmup=2):
    """The headline grid split into z-slabs on one GPU (slabs.SlabGrid): the
    same step through the halo pack/unpack kernels and the dt minimum over
    the slabs; zone-updates/s, the exchange time, and whether its first step
    equals the undivided grid's bit for bit."""
    import torch
    from paper_2211_13295_gb300 import slabs
    sg = slabs.SlabGrid(prob, parts)
    sg.set_state(Uh.numpy())
    same = None
    if U1 is not None:
        dt0 = sg.cfl_dt()
        sg.step(dt0, sync=True)
        same = bool(np.array_equal(sg.get_state(), U1))
        sg.set_state(Uh.numpy())
        sg.set_time(0.0)
    sg.cfl_dt()
    for _ in range(warmup):
        sg.step(0.0, sync=False)
    torch.cuda.synchronize()
    sg.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        sg.step(0.0, sync=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = sg.profile_read()
    sg.check()
    sg.close()
    return {"slabs": parts, "value": prob.zones / (ms * 1e-3), "unit": "zone-updates/s", "ms_per_step": ms,
            "exchange_ms_per_step": prof["halo_exchange"][1] / steps,
            "first_step_bitwise_equal_to_undivided": same}


def run_native(args, rank, world, local):
    import torch
    from paper_2211_13295_gb300 import awe, build, opcount
    from paper_2211_13295_gb300 import problems as P
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        # one grid of n x n x (n * world) zones split into z-slabs, one n^3
        # slab per GPU: per step one halo exchange (NCCL point-to-point) and
        # one all-reduce MIN of dt (weak scaling: fixed work per GPU)
        from paper_2211_13295_gb300 import slabs
        gprob = P.tgv3d(n=args.n, order=args.order, cfl=0.3, nz=args.n * world)
        grid = slabs.DistSlabGrid(gprob, rank, world, prec=args.form, gate=False)
        prob = grid.sub_prob
        Uh = gpu_state(prob)
    else:
        gprob = prob = workload(args.n, args.order)
        Uh = gpu_state(prob)
        grid = awe.Grid(prob, prec=args.form, gate=args.gate)
    if args.gate:
        from paper_2211_13295_gb300.gate_train import he_init
        grid.gate_set_weights(he_init(awe.gate_dims(prob.dim, prob.order)[0], 2211))
    grid.set_state(Uh.numpy())
    # one explicit step from the initial state for the stated error
    dt0 = grid.cfl_dt()
    grid.step(dt0)
    grid.check()
    U1 = grid.get_state() if rank == 0 and world == 1 and not args.no_cpu else None
    grid.set_state(Uh.numpy())
    grid.set_time(0.0)

    clk = Clocks(local)
    ms, prof = time_steps(grid, args.steps, args.warmup, world)
    clocks = clk.stop()
    ms = max_over_ranks(ms, world)
    zones = prob.zones
    value = world * zones * args.steps / (ms * 1e-3)

    # dominant kernel: the predictor (FP64 pipe)
    n_pred, ms_pred = prof["predictor"]
    avg_pred = ms_pred / max(n_pred, 1)
    flops_pred = opcount.predictor_flops_per_launch(prob)
    achieved = flops_pred / (avg_pred * 1e-3) / 1e12
    # DRAM bytes of one predictor launch: not measurable inside this run (ncu
    # replays kernels); taken from one ncu capture of the same kernel on a
    # 48^3 grid, scaled to this launch by the box zones it processes, and
    # labelled as such in the line
    traffic, traffic_source = None, None
    tr_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_file) and prob.order == 4:
        tr = json.load(open(tr_file))
        key = "predictor_fp64_per_launch" if args.form == "fp64" else "predictor_fp32_per_launch"
        if tr.get(key) is not None and tr.get(key + "_kernel_sha") == opcount.predictor_source_sha():
            traffic = tr[key]
            traffic_source = tr.get(key + "_source")
    launches_per_step = sum(v[0] for v in prof.values()) / max(args.steps, 1)
    # kernel launches of the timed region: profiled spans + 1 finalize per step
    gpu_launches = int(round(sum(v[0] for k, v in prof.items() if k != "halo_exchange") + args.steps))
    if world > 1:
        # per exchange two pack and two unpack kernels (their ghost fills are
        # profiled spans already)
        gpu_launches += 4 * prof["halo_exchange"][0]

    grid.set_state(Uh.numpy())
    grid.cfl_dt()
    e2e_ms = max_over_ranks(time_e2e(grid, Uh, max(1, min(args.steps, 3)), world), world)
    e2e_steps = max(1, min(args.steps, 3))
    nbytes = Uh.numel() * 8
    grid.close()

    forms = {}
    run_forms = not args.no_forms and args.form == "fp64" and world == 1
    if run_forms:
        g32 = awe.Grid(prob, prec="fp32")
        g32.set_state(Uh.numpy())
        dtf = g32.cfl_dt()
        g32.step(dtf)
        U1f = g32.get_state() if U1 is not None else None
        g32.set_state(Uh.numpy())
        ms32, prof32 = time_steps(g32, args.steps, args.warmup, world)
        ms32 = max_over_ranks(ms32, world)
        np32, mp32 = prof32["predictor"]
        g32.close()
        f32 = {"value": world * zones * args.steps / (ms32 * 1e-3), "ms_per_step": ms32 / args.steps,
               "dtype": "f32 bulk, f64 update/WENO epsilon path/CFL",
               "predictor_ms": mp32 / max(np32, 1),
               "predictor_tflops": flops_pred / (mp32 / max(np32, 1) * 1e-3) / 1e12,
               "predictor_frac_fp32_peak": flops_pred / (mp32 / max(np32, 1) * 1e-3) / 1e12 / PEAK_FP32}
        if U1f is not None:
            sc = np.abs(U1[0]).sum()
            f32["rel_l1_vs_fp64_gpu_one_step"] = max(
                float(np.abs(U1f[v] - U1[v]).sum() / max(np.abs(U1[v]).sum(), sc)) for v in range(5))
            sci = np.abs(U1[0]).max()
            f32["rel_linf_vs_fp64_gpu_one_step"] = max(
                float(np.abs(U1f[v] - U1[v]).max() / max(np.abs(U1[v]).max(), sci)) for v in range(5))
        f32["stage_ms_per_step"] = {k: round(v[1] / args.steps, 3) for k, v in prof32.items() if v[0]}
        forms["fp32_bulk"] = f32

    if run_forms:
        forms.update(gated_forms(args, prob, Uh, U1, zones, world))
        gate_params = forms.pop("_params")

    table2 = table4 = solvers = small = others = slab1 = None
    if run_forms:
        slab1 = slab_decomposition_1gpu(prob, Uh, U1)
        small = small_grid_graph()
        others = other_configs(world, gate_params)
        table2 = orders_192(args, world)
        table4 = orders_192(args, world, scheme="ssprk")
        solvers = {k: orders_192(args, world, riemann=k, orders=(4,))["O4"] for k in ("hll", "hllem", "rusanov")}
        rk_gated = orders_192(args, world, scheme="ssprk", orders=(4,), gate=gate_params)["O4"]
        table4["O4_gated"] = rk_gated

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, parity = cpu_baseline_and_parity(prob, U1, Uh.numpy(), dt0)

    peak = PEAK_FP64 if args.form == "fp64" else PEAK_FP32
    # the same kernel against the HBM roofline: its measured DRAM bytes per
    # launch (ncu, profiles/traffic.json) over its CUDA-event launch time
    hpk, hsrc = hbm_peak()
    hbm_line = None
    if traffic is not None and args.form == "fp64":
        gbs = traffic / (avg_pred * 1e-3) / 1e9
        hbm_line = {"achieved_gbs": gbs, "peak_gbs": hpk, "frac": gbs / hpk, "peak_source": hsrc,
                    "step_state_bytes": 2 * nbytes,
                    "note": "FP64-pipe bound: DRAM traffic is a small fraction of the HBM roofline"}
    if rank == 0:
        line = {
            "metric": "zone-updates/sec per full ADER-WENO step at stated L1 error vs FP64 oracle",
            "value": value,
            "unit": "zone-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.form == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(gprob), "n": prob.n[0], "order": prob.order,
                       "form": args.form, "riemann": "hllc",
                       "parallelism": "one grid" if world == 1 else
                       f"z-slabs x{world}: one {args.n}^3 slab per GPU, halo exchange + dt MIN per step",
                       "l2": "inputs larger than L2 (state 671 MB, modes 13.7 GB per step)",
                       "l1_vs_oracle_one_step": parity},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_source,
                         "kernel": "predictor (" + ("k_predict_direct" if prob.order != 4 else
                                                    "k_predict_fact<double>" if args.form == "fp64" else
                                                    "k_predict_lines (FP32)") + ")",
                         "peak_source": f"derived: 152 SMs x {'2 FP64' if args.form == 'fp64' else '128 FP32'} FMA/clk x 2 x 2.07 GHz",
                         "algorithmic_flops_per_launch": flops_pred, "avg_launch_ms": avg_pred,
                         "hbm": hbm_line},
            "stage_ms_per_step": {k: v[1] / args.steps for k, v in prof.items() if v[0]},
            "clocks": clocks,
            "e2e": {"value": world * zones * e2e_steps / (e2e_ms * 1e-3), "unit": "zone-updates/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": gpu_launches,
            "cpu_baseline": cpu,
            "forms": forms,
            "orders_tgv192_fp64": table2,
            "ssprk_orders_tgv192_fp64": table4,
            "riemann_tgv192_o4_fp64": solvers,
            "small_grid_cuda_graph": small,
            "slab_decomposition_1gpu": slab1,
            "other_workloads": others,
        }
        if world > 1:
            line["halo_exchange_ms_per_step"] = prof.get("halo_exchange", (0, 0.0))[1] / args.steps
            line["comm_nranks"] = world
        # last key: a compact digest of every form and workload, so that the
        # end of the line (what a log tail keeps) carries all the numbers
        line["summary"] = summary(line)
        print(json.dumps(line))


def _sig(x, k=3):
    if x is None:
        return None
    if isinstance(x, (int, float)) and x != 0 and math.isfinite(x):
        return float(f"{x:.{k}g}")
    return x


def summary(line):
    """value (zone-updates/s), ms per step, predictor roofline fraction and
    one-step errors of each form; status of the other workloads"""
    out = {"fp64": {"v": _sig(line["value"]), "ms": _sig(line["ms_per_step"]),
                    "frac": _sig(line["roofline"]["frac"]),
                    "l1_oracle": _sig(line["config"].get("l1_vs_oracle_one_step"))}}
    forms = line.get("forms") or {}
    if "fp32_bulk" in forms:
        f = forms["fp32_bulk"]
        out["fp32"] = {"v": _sig(f["value"]), "ms": _sig(f["ms_per_step"]),
                       "frac": _sig(f["predictor_frac_fp32_peak"]),
                       "l1": _sig(f.get("rel_l1_vs_fp64_gpu_one_step")),
                       "linf": _sig(f.get("rel_linf_vs_fp64_gpu_one_step"))}
    for k in ("fp64_gated", "fp32_gated"):
        if k in forms:
            f = forms[k]
            out[k] = {"v": _sig(f["value"]), "ms": _sig(f["ms_per_step"]),
                      "flagged": _sig(f["flagged_fraction"]),
                      "l1_full_weno": _sig(f.get("rel_l1_vs_full_weno_fp64_one_step"))}
    for name, d in (line.get("other_workloads") or {}).items():
        out[name.split("_")[0]] = {"v": _sig(d["value"]), "ms": _sig(d["ms_per_step"]),
                                   "status": "ok" if d["status"] == "ok" else d["status"][:40]}
    return out


def run_reference(args, rank, world):
    """The FP64 oracle as the reference arm: each step is one oracle step of the
    same workload on a bounded sample (a periodic 24^3 Taylor-Green grid of
    the workload's order, FP64, HLLC), on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2211_13295_gb300 import problems as P
    small = P.tgv3d(n=24, order=args.order, cfl=0.3)
    U = small.initial_state()
    orc = oracle.Oracle(small)
    dt = orc.cfl_dt(U, small.cfl)
    t = 0.0
    for _ in range(args.warmup):
        U, smax, _ = orc.step(U, t, dt)
        t += dt
        dt = small.cfl / smax
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, smax, _ = orc.step(U, t, dt)
        t += dt
        dt = small.cfl / smax
    el = time.perf_counter() - t0
    value = small.zones * args.steps / el
    line = {
        "impl": "reference",
        "metric": "zone-updates/sec per full ADER-WENO step at stated L1 error vs FP64 oracle",
        "value": value, "unit": "zone-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(workload(args.n, args.order)),
                   "sample": f"tgv3d 24^3 order {args.order} per step"},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "tgv3d 24^3 order 4 FP64, one oracle step per bench step"},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
