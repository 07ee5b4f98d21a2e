"""Throughput benchmark of the pointwise thermochemistry hot path on GB300.

One step = one pass of the whole path over one batch resident in HBM: the
temperature from internal energy by Newton iteration, then species thermo,
rate and equilibrium constants, rates of progress and net production rates,
on the synthetic 53-species / 325-reaction mechanism at 2^22 states (FP64).
The batch (1.85 GB of inputs) is far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun with one rank per GPU; each rank evaluates its own
2^22 states (points are independent: weak scaling, no collective on the data
path); the step time is the maximum over ranks.  --impl reference times the CPU
oracle on the host cores on bounded samples of the same workload.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "state-evals/sec (T solve + omega_k, FP64)"
CONFIG_INDEX = 1
# FP64 pipe of GB300: 2 DFMA lanes per SM per clock (measured by a DFMA
# microbenchmark: 2.07 lanes/SM/clk).  The SM count is read from the device and
# the maximum SM clock from nvidia-smi (clocks.max.sm) at run time; the values
# below (152 SMs, 2070 MHz: 1258.6 GFLOP/s) are used only where they cannot be read.
FP64_LANES_PER_SM = 2
N_SM_DEFAULT = 152
SM_MAX_MHZ_DEFAULT = 2070.0
FP64_PEAK_GFLOPS = 2.0 * FP64_LANES_PER_SM * N_SM_DEFAULT * SM_MAX_MHZ_DEFAULT / 1e3   # DFMA = 2 flops


def fp64_peak_gflops(n_sm: int, sm_max_mhz: float) -> float:
    return 2.0 * FP64_LANES_PER_SM * n_sm * sm_max_mhz / 1e3


def sm_max_mhz_of(gpu_index: int) -> float:
    """clocks.max.sm of the GPU from nvidia-smi (MHz), else the GB300 default."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        v = float(out.stdout.strip().splitlines()[0])
        return v if v > 0 else SM_MAX_MHZ_DEFAULT
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return SM_MAX_MHZ_DEFAULT

# DRAM traffic of one launch of the timed kernel, from an ncu capture of this
# kernel source (hash of the emitted source); None once the kernel changes.
PROFILED_TRAFFIC = {
    # 2^19-state ncu captures scaled by 8 to a 2^22-state launch
    "953a6879ca9d63b7": 3.334e9,
    "a24d27e8509fd73d": 3.330e9,
    # 2^20-state capture (dram__bytes_read.sum + dram__bytes_write.sum) scaled by 4
    "d480c6fd1d99f5f7": 3.497e9,
}


def _dist():
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
        return dist
    return None


def rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def max_over_ranks(x: float, device=None) -> float:
    dist = _dist()
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    dist = _dist()
    if dist is not None:
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = tempfile.TemporaryFile(mode="w+")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        load = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def workload_config(n: int) -> dict:
    cfg = {"workload": "synthetic GRI-sized mechanism, 53 species / 325 reactions (30 third-body, 25 Troe, "
                       "28 duplicate pairs); %d states/step; T from internal energy by Newton + omega_k" % n,
           "mechanism_seed": 2503 + CONFIG_INDEX, "state_seed": 24286 + CONFIG_INDEX,
           "T_K": [300, 2800], "p_atm": [0.5, 20], "Y": "Dirichlet(0.5)",
           "n_points": n, "layout": "SoA [species][point] FP64",
           "l2": "inputs 1.85 GB/step > 129 MB L2 (no flush needed)"}
    return cfg


def cpu_oracle_rate(path: str, n: int, seed_offset: int = 0):
    """States/s of the CPU oracle (T solve + omega) on an n-point sample of the workload."""
    from oracle import oracle as O
    from paper_2503_24286_gb300 import synth
    O.build()
    orc = O.Oracle(path)
    st = synth.config_states(CONFIG_INDEX, n=n, offset_seed=100 + seed_offset)
    rho = orc.density(st.p, st.T, st.Y)
    e = orc.internal_energy(st.T, st.Y)
    t0 = time.perf_counter()
    T, _, _ = orc.temperature(e, st.Y)
    orc.net_production_rates(rho, T, st.Y)
    dt = time.perf_counter() - t0
    return n / dt, O.threads(), dt


def cpu_oracle_rate_one_core(path: str, n: int):
    """The same on one host core (OpenMP limited to one thread for the call)."""
    from oracle import oracle as O
    O.build()
    prev = O.threads()
    O.set_threads(1)
    try:
        rate, _, dt = cpu_oracle_rate(path, n, seed_offset=7)
    finally:
        O.set_threads(prev)
    return rate, dt


def run_reference(args):
    rank, world = rank_world()
    if rank != 0:
        return 0
    from paper_2503_24286_gb300 import synth
    d = tempfile.mkdtemp()
    path = os.path.join(d, "mech.txt")
    synth.write_mechanism(synth.config_mechanism(CONFIG_INDEX), path)
    n = args.ref_sample
    for i in range(args.warmup):
        cpu_oracle_rate(path, min(n, 4096), i)
    times = []
    cores = 1
    for i in range(args.steps):
        rate, cores, dt = cpu_oracle_rate(path, n, 1000 + i)
        times.append(dt)
    tot = sum(times)
    value = n * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "states/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(n),
            "cpu_baseline": {"value": value, "unit": "states/s", "cores": cores, "kind": "oracle",
                             "sample": "%d states per step of the same workload (seeded), plain FP64 C++ oracle, "
                                       "OpenMP over points" % n},
            "e2e": {"value": value, "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0



def derivative_rates(mech, synth, dev, stream, args, rank):
    """Jacobian-evals/s and JVP/VJP states/s on 2^20 resident states of the same mechanism."""
    import torch
    mech.prepare("all")
    n = args.deriv_points
    cfg = synth.CONFIGS[2]
    T, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 2 + 7919 * rank, dev)
    rho = mech.density(p, T, Y)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    d_rho = torch.randn(n, dtype=torch.float64, device=dev, generator=g) * rho * 1e-3
    d_T = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    d_Y = torch.randn((53, n), dtype=torch.float64, device=dev, generator=g) * 1e-4
    w_bar = torch.randn((53, n), dtype=torch.float64, device=dev, generator=g)
    J = torch.empty((54 * 54, n), dtype=torch.float64, device=dev)
    out = torch.empty((53, n), dtype=torch.float64, device=dev)
    calls = {
        "jvp": lambda: mech.jvp(rho, T, Y, d_rho, d_T, d_Y, out=out),
        "vjp": lambda: mech.vjp(rho, T, Y, w_bar),
        "jacobian": lambda: mech.jacobian(rho, T, Y, out=J),
        "omega_isothermal": lambda: mech.net_production_rates(rho, Y, T=T, out=out),
    }
    res = {"workload": "same mechanism, %d states, T ~ U[300, 2800] K, p ~ U[0.5, 20] atm, Dirichlet Y; "
                       "Jacobian d(Tdot, omega)/d(T, Y) at fixed rho, [(N+1)^2][n] = %.1f GB out" % (n, 54 * 54 * 8 * n / 1e9)}
    steps = max(2, min(args.steps, 5))
    for name, f in calls.items():
        for _ in range(3):
            f()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            f()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
        res[name + "_ms"] = ms
        res[name + "_per_s"] = n / (ms * 1e-3)
    res["jacobian_out_GB_per_s"] = 54 * 54 * 8 * n / (res["jacobian_ms"] * 1e-3) / 1e9
    # FP64 roofline of each derivative kernel: the emitter's static FP64 flops per
    # state x states/s, against the FP64 peak (Jacobian-evals/s vs FP64 roofline)
    for name, key in (("jvp", "jvp_fp64_flops_per_point"), ("vjp", "vjp_fp64_flops_per_point"),
                      ("jacobian", "jacobian_fp64_flops_per_point"),
                      ("omega_isothermal", "omega_fp64_flops_per_point")):
        f = mech.stat(key)
        res[name + "_fp64_flops_per_state_static"] = f
        res[name + "_gflops"] = f * res[name + "_per_s"] / 1e9
        res[name + "_frac"] = f * res[name + "_per_s"] / (args.fp64_peak * 1e9)
    del J
    return res



def learned_guess_rates(mech, path, synth, dev, stream, args, rank):
    """Train the guess network on 2^24 states, then time the temperature solve on 2^22
    held-out states with the fixed 1200 K guess and with the learned guess, in the
    library's default (FP32 then FP64) and the paper's FP64-only Newton."""
    import time as _t
    import torch
    from paper_2503_24286_gb300 import binding as B
    cfg = synth.CONFIGS[3]
    res = {"workload": "train %d states (T ~ U[300, 2800] K, Dirichlet Y, e by the library's energy kernel), "
                       "infer %d held-out states; MLP 54-64-64-1 SiLU, BF16 tensor-core inference"
                       % (args.train_points, args.points)}
    T, p, Y = synth.generate_states_torch(53, args.train_points, cfg["T"], cfg["p_atm"],
                                          synth.STATE_SEED_BASE + 3 + 7919 * rank, dev)
    del p
    torch.cuda.synchronize(dev)
    t0 = _t.perf_counter()
    loss = mech.mlp_train(T, Y, "epochs=1;batch=1024;lr=1e-2;seed=1")
    res["train_s"] = _t.perf_counter() - t0
    res["train_final_loss"] = loss
    del T, Y
    T, p, Y = synth.generate_states_torch(53, args.points, cfg["T"], cfg["p_atm"],
                                          synth.STATE_SEED_BASE + 3 + 104729 + 7919 * rank, dev)
    e = mech.internal_energy(T, Y)
    _, Tg = mech.mlp_guess(e, Y)
    res["guess_rms_K"] = float(((Tg - T) ** 2).mean().sqrt().item())
    out = torch.empty_like(T)
    f = os.path.join(os.path.dirname(path), "guess.bin")
    mech.mlp_save(f)
    m64 = B.Mechanism(path, "newton=fp64")
    m64.mlp_load(f)
    steps = max(2, min(args.steps, 5))
    for tag, m in (("newton_mixed", mech), ("newton_fp64", m64)):
        r = {}
        for guess in ("fixed", "learned"):
            learned = guess == "learned"
            _, it = m.temperature(e, Y, learned=learned, with_iters=True)
            r[guess + "_iters_mean"] = float(it.double().mean().item())
            for _ in range(3):
                m.temperature(e, Y, learned=learned, out=out)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                m.temperature(e, Y, learned=learned, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
            r[guess + "_ms"] = ms
            r[guess + "_states_per_s"] = args.points / (ms * 1e-3)
            assert (torch.abs(out - T) / T).max().item() < 1e-10
        res[tag] = r
    return res



def large_mechanism_path(synth):
    d = tempfile.mkdtemp()
    path = os.path.join(d, "mech4.txt")
    synth.write_mechanism(synth.config_mechanism(4), path)
    return path


def start_large_compile(path):
    """Compile the large mechanism's derivative groups (NVRTC, written to the
    on-disk kernel cache) in a host thread on a compile-only handle, so the
    minutes of compilation overlap the other rows; join() before the rows that
    need them and before any CPU timing."""
    import threading
    from paper_2503_24286_gb300 import binding as B
    err = []

    def run():
        try:
            B.Mechanism(path, "device=0").prepare("jvp,vjp")
            B.Mechanism(path, "device=0;variant=warp").prepare("jvp,vjp,jacobian,jacobian_adiabatic")
        except Exception as e:  # reported by the rows that need the groups
            err.append(repr(e))
    t = threading.Thread(target=run, daemon=True)
    t.start()
    return t, err


def large_mechanism_rates(path, synth, dev, stream, args, rank):
    """160 species / 1100 reactions at 2^21 states: T from e + omega, and the JVP and
    VJP (intermediates recomputed, nothing stored), each with one thread per state
    (emitted straight-line code, species arrays in a global scratch) against one
    warp per state (lanes split the reactions); also the warp variant of the
    forward on the 53-species workload.  Each row with its FP64 roofline fraction
    (emitter's static FP64 flops per state)."""
    import torch
    from paper_2503_24286_gb300 import binding as B
    cfg = synth.CONFIGS[4]
    n = args.large_points
    res = {"workload": "synthetic 160 species / 1100 reactions (80 third-body, 60 Troe), %d states, "
                       "T ~ U[300, 2800] K, p ~ U[1, 40] atm; T from e + omega, JVP and VJP (unit-scale random "
                       "seed vectors)" % n}
    mt = B.Mechanism(path)
    mw = B.Mechanism(path, "variant=warp")
    T, p, Y = synth.generate_states_torch(160, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 4 + 7919 * rank, dev)
    rho = mt.density(p, T, Y)
    e = mt.internal_energy(T, Y)
    del p
    w = torch.empty((160, n), dtype=torch.float64, device=dev)
    To = torch.empty(n, dtype=torch.float64, device=dev)
    steps = max(2, min(args.steps, 5))

    def timed(f):
        for _ in range(3):
            f()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            f()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1) / steps, dev)

    peak = args.fp64_peak * 1e9
    f_fwd = mt.stat("omega_fp64_flops_per_point") + 2 * mt.stat("tsolve_collapse_fp64_ops") + \
        3 * 2 * mt.stat("tsolve_iter_fp64_ops_mixed")
    res["fp64_flops_per_state_static"] = f_fwd
    for tag, m in (("thread_per_state", mt), ("warp_per_state", mw)):
        ms = timed(lambda: m.net_production_rates(rho, Y, e=e, T_out=To, out=w))
        res[tag + "_ms"] = ms
        res[tag + "_states_per_s"] = n / (ms * 1e-3)
        res[tag + "_frac"] = f_fwd * n / (ms * 1e-3) / peak
        assert m.nonconverged() == 0
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    d_rho = torch.randn(n, dtype=torch.float64, device=dev, generator=g) * rho * 1e-3
    d_T = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
    d_Y = torch.randn((160, n), dtype=torch.float64, device=dev, generator=g) * 1e-4
    w_bar = torch.randn((160, n), dtype=torch.float64, device=dev, generator=g)
    args.large_compile.join()
    deriv = {}
    for tag, m in (("thread_per_state", mt), ("warp_per_state", mw)):
        try:
            if tag == "warp_per_state" and m.stat("deriv_warp_per_state") <= 0:
                deriv[tag] = {"unavailable": "no warp-per-state derivative kernels for this mechanism"}
                continue
            m.prepare("jvp,vjp")
        except B.PyroError as ex:
            deriv[tag] = {"unavailable": str(ex)}
            continue
        r = {}
        for name, f, key in (("jvp", lambda: m.jvp(rho, T, Y, d_rho, d_T, d_Y, out=w), "jvp_fp64_flops_per_point"),
                             ("vjp", lambda: m.vjp(rho, T, Y, w_bar), "vjp_fp64_flops_per_point")):
            ms = timed(f)
            fl = m.stat(key)
            r[name + "_ms"] = ms
            r[name + "_states_per_s"] = n / (ms * 1e-3)
            r[name + "_fp64_flops_per_state_static"] = fl
            r[name + "_frac"] = fl * n / (ms * 1e-3) / peak
        deriv[tag] = r
    res["derivatives"] = deriv
    # dense Jacobians, one block of 8 warps per state (variant=warp), on --large-jac-points
    # states; FP64 fraction against the thread-per-state kernel's static count of the same
    # quantity (the algorithmic operations of the assembly)
    del d_Y, w_bar, w
    nj = args.large_jac_points
    jac = {"states": nj}
    if mw.stat("jacobian_cta") > 0:
        rj, Tj, Yj = rho[:nj].contiguous(), T[:nj].contiguous(), Y[:, :nj].contiguous()
        mw.prepare("jacobian,jacobian_adiabatic")
        J = torch.empty((161 * 161, nj), dtype=torch.float64, device=dev)
        ms = timed(lambda: mw.jacobian(rj, Tj, Yj, out=J))
        fl = mt.stat("jacobian_fp64_flops_per_point")
        jac.update(jacobian_ms=ms, jacobian_states_per_s=nj / (ms * 1e-3), jacobian_out_GB_per_s=J.numel() * 8 / (ms * 1e6),
                   jacobian_fp64_flops_per_state_static=fl, jacobian_frac=fl * nj / (ms * 1e-3) / peak)
        del J
        Ja = torch.empty((160 * 160, nj), dtype=torch.float64, device=dev)
        ms = timed(lambda: mw.jacobian_adiabatic(rj, Tj, Yj, out=Ja))
        fl = mt.stat("jacobian_adiabatic_fp64_flops_per_point")
        jac.update(jacobian_adiabatic_ms=ms, jacobian_adiabatic_states_per_s=nj / (ms * 1e-3),
                   jacobian_adiabatic_fp64_flops_per_state_static=fl,
                   jacobian_adiabatic_frac=fl * nj / (ms * 1e-3) / peak)
        del Ja
    else:
        jac["unavailable"] = "no block-per-state Jacobian kernels for this mechanism"
    res["jacobian_block_per_state"] = jac
    return res


def large_derivative_rates(path, synth, dev, stream, args, rank):
    """The Jacobian-type kernels on the 160-species mechanism (rows from tables,
    species arrays in the global scratch): dense 161 x 161 Jacobian and dS/dY at
    fixed (rho, e) on 2^15 states, one Crank-Nicolson step of 2^14 states at
    dt = 1e-46 s (sizes: --large-deriv-points and half of it).  Off by default
    (the three units take minutes to compile)."""
    import torch
    from paper_2503_24286_gb300 import binding as B
    parts = args.large_derivatives.split(",")
    m = B.Mechanism(path)
    m.prepare(args.large_derivatives)
    cfg, ccfg = synth.CONFIGS[4], synth.CONFIGS[8]
    n, nc = args.large_deriv_points, args.large_deriv_points // 2
    res = {"workload": "160 species / 1100 reactions; Jacobian and dS/dY on %d states (T ~ U[300, 2800] K), "
                       "Crank-Nicolson on %d states (T ~ U[2000, 2800] K, dt = 1e-46 s); timed: %s"
                       % (n, nc, args.large_derivatives)}
    T, p, Y = synth.generate_states_torch(160, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 4 + 7919 * rank, dev)
    rho = m.density(p, T, Y)

    def timed(fn, steps=3):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1) / steps, dev)

    if "jacobian" in parts:
        J = torch.empty((161 * 161, n), dtype=torch.float64, device=dev)
        ms = timed(lambda: m.jacobian(rho, T, Y, out=J))
        res.update(jacobian_ms=ms, jacobian_per_s=n / (ms * 1e-3), jacobian_out_GB_per_s=J.numel() * 8 / (ms * 1e6))
        del J
    if "jacobian_adiabatic" in parts:
        Ja = torch.empty((160 * 160, n), dtype=torch.float64, device=dev)
        ms = timed(lambda: m.jacobian_adiabatic(rho, T, Y, out=Ja))
        res.update(jacobian_adiabatic_ms=ms, jacobian_adiabatic_per_s=n / (ms * 1e-3))
        del Ja
    if "cn" not in parts:
        return res
    T, p, Y = synth.generate_states_torch(160, nc, ccfg["T"], ccfg["p_atm"], synth.STATE_SEED_BASE + 8 + 7919 * rank, dev)
    rho = m.density(p, T, Y)
    To, Yo = torch.empty_like(T), torch.empty_like(Y)
    last = []
    ms = timed(lambda: last.append(m.cn_step(ccfg["dt"], rho, T, Y, T_out=To, Y_out=Yo, with_iters=True)[2]), steps=2)
    torch.cuda.synchronize(dev)
    it = last[-1]
    res.update(cn_step_ms=ms, cn_step_per_s=nc / (ms * 1e-3), newton_iters_mean=float(it.float().mean().item()),
               newton_iters_max=int(it.max().item()), cn_failed=int((it < 0).sum().item()))
    return res


def crank_nicolson_rates(synth, dev, stream, args, rank):
    """One Crank-Nicolson step (Sec. A.3.2) of 2^18 states of the 53-species
    mechanism at T ~ U[2000, 2800] K with dt = 3e-41 s (the synthetic kinetics'
    stiff time scale), and the chemical Jacobian dS/dY at fixed (rho, e) on the
    same states."""
    import torch
    from paper_2503_24286_gb300 import binding as B
    d = tempfile.mkdtemp()
    path = os.path.join(d, "mech.txt")
    cfg = synth.CONFIGS[5]
    synth.write_mechanism(synth.config_mechanism(5), path)
    m = B.Mechanism(path)
    m.prepare("jacobian_adiabatic,cn")
    n = args.cn_points
    T, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 5 + 7919 * rank, dev)
    rho = m.density(p, T, Y)
    del p
    dt = cfg["dt"]
    res = {"workload": "53 species / 325 reactions, %d states, T ~ U[2000, 2800] K, p ~ U[0.5, 20] atm, "
                       "Dirichlet Y; one Crank-Nicolson step, dt = %g s, Newton tol 1e-12 on max|dY|; "
                       "Newton matrix by FP32 LU + 1 FP64 refinement step" % (n, dt)}
    To = torch.empty_like(T)
    Yo = torch.empty_like(Y)
    _, _, it = m.cn_step(dt, rho, T, Y, T_out=To, Y_out=Yo, with_iters=True)
    torch.cuda.synchronize(dev)
    assert m.nonconverged() == 0 and (it > 0).all().item()
    res["newton_iters_mean"] = float(it.double().mean().item())
    res["newton_iters_max"] = int(it.max().item())
    # chord variant: the first iterate's factorisation kept for the whole step
    mc = B.Mechanism(path, "cn_newton=chord")
    mc.prepare("cn")
    _, _, itc = mc.cn_step(dt, rho, T, Y, T_out=To, Y_out=Yo, max_newton=60, with_iters=True)
    torch.cuda.synchronize(dev)
    assert mc.nonconverged() == 0 and (itc > 0).all().item()
    res["chord_newton_iters_mean"] = float(itc.double().mean().item())
    res["chord_newton_iters_max"] = int(itc.max().item())
    steps = max(2, min(args.steps, 3))
    J = torch.empty((53 * 53, n), dtype=torch.float64, device=dev)
    calls = {"cn_step": lambda: m.cn_step(dt, rho, T, Y, T_out=To, Y_out=Yo),
             "cn_step_chord": lambda: mc.cn_step(dt, rho, T, Y, T_out=To, Y_out=Yo, max_newton=60),
             "jacobian_adiabatic": lambda: m.jacobian_adiabatic(rho, T, Y, out=J)}
    for name, f in calls.items():
        f()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            f()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
        res[name + "_ms"] = ms
        res[name + "_per_s"] = n / (ms * 1e-3)
    del J
    return res


def pressure_dependent_rates(synth, dev, stream, args, rank):
    """T from e + omega_k on 2^22 states of the 53-species variant with 10 SRI
    falloff and 20 PLOG reactions (same kernel design as the headline)."""
    import torch
    from paper_2503_24286_gb300 import binding as B
    d = tempfile.mkdtemp()
    path = os.path.join(d, "mech7.txt")
    cfg = synth.CONFIGS[7]
    synth.write_mechanism(synth.config_mechanism(7), path)
    m = B.Mechanism(path)
    n = args.pdep_points
    T, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 7 + 7919 * rank, dev)
    rho = m.density(p, T, Y)
    e = m.internal_energy(T, Y)
    del p
    w = torch.empty((53, n), dtype=torch.float64, device=dev)
    To = torch.empty(n, dtype=torch.float64, device=dev)
    for _ in range(3):
        m.net_production_rates(rho, Y, e=e, T_out=To, out=w)
    torch.cuda.synchronize(dev)
    assert m.nonconverged() == 0
    steps = max(2, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        m.net_production_rates(rho, Y, e=e, T_out=To, out=w)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    flops = m.stat("omega_fp64_flops_per_point") + 2 * m.stat("tsolve_collapse_fp64_ops") + \
        3 * 2 * m.stat("tsolve_iter_fp64_ops_mixed")
    return {"workload": "53 species / 325 reactions with 10 SRI falloff and 20 PLOG (3-5 nodes in [0.1, 100] atm) "
                        "reactions, %d states, T ~ U[300, 2800] K, p ~ U[0.5, 20] atm; T from e + omega" % n,
            "ms": ms, "states_per_s": n / (ms * 1e-3), "fp64_flops_per_state_static": flops,
            "fp64_frac": flops * n / (ms * 1e-3) / (args.fp64_peak * 1e9)}


def transport_rates(mech, synth, dev, stream, args, rank):
    """Mixture-averaged mu, kappa and D_km (Sec. A.2) on 2^20 resident states of the
    53-species mechanism (T ~ U[300, 2800] K, Dirichlet Y)."""
    import torch
    mech.prepare("transport")
    n = args.transport_points
    cfg = synth.CONFIGS[1]
    T, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 1 + 17 + 7919 * rank, dev)
    del p
    mu = torch.empty(n, dtype=torch.float64, device=dev)
    ka = torch.empty(n, dtype=torch.float64, device=dev)
    Dm = torch.empty((53, n), dtype=torch.float64, device=dev)
    from paper_2503_24286_gb300 import binding as B

    def call():
        B._check(B.lib().pyro_transport(mech.handle, n, *[B._ptr(a)[0] for a in (T, Y, mu, ka, Dm)],
                                        B._stream([T])))
    for _ in range(3):
        call()
    torch.cuda.synchronize(dev)
    steps = max(2, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    ops = mech.stat("transport_fp64_ops_per_point")
    return {"workload": "53 species, %d states, T ~ U[300, 2800] K, Dirichlet Y; mu (Wilke), kappa, D_km" % n,
            "ms": ms, "states_per_s": n / (ms * 1e-3),
            "fp64_ops_per_state_static": ops,
            "fp64_pipe_frac": ops * n / (ms * 1e-3) / (args.fp64_peak * 1e9 / 2)}


def run_rows_only(args):
    """--only ROWS: run just the named secondary rows (for profiling one kernel
    family under ncu without the headline launches before it) and print one JSON
    line with those rows; no headline value."""
    import torch
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    from paper_2503_24286_gb300 import synth
    rank, _ = rank_world()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    BLD.build()
    args.fp64_peak = fp64_peak_gflops(torch.cuda.get_device_properties(dev).multi_processor_count,
                                      sm_max_mhz_of(local))
    rows = set(args.only.split(","))
    stream = torch.cuda.current_stream(dev)
    d = tempfile.mkdtemp()
    path = os.path.join(d, "mech.txt")
    synth.write_mechanism(synth.config_mechanism(CONFIG_INDEX), path)
    out = {}
    if "large" in rows:
        path4 = large_mechanism_path(synth)
        args.large_compile, _ = start_large_compile(path4)
        out["large_mechanism"] = large_mechanism_rates(path4, synth, dev, stream, args, rank)
    mech = B.Mechanism(path) if rows & {"derivatives", "learned", "transport"} else None
    if "derivatives" in rows:
        out["derivatives"] = derivative_rates(mech, synth, dev, stream, args, rank)
    if "learned" in rows:
        out["learned_guess"] = learned_guess_rates(mech, path, synth, dev, stream, args, rank)
    if "pdep" in rows:
        out["pressure_dependent"] = pressure_dependent_rates(synth, dev, stream, args, rank)
    if "transport" in rows:
        out["transport"] = transport_rates(mech, synth, dev, stream, args, rank)
    if "cn" in rows:
        out["crank_nicolson"] = crank_nicolson_rates(synth, dev, stream, args, rank)
    if rank == 0:
        print(json.dumps({"rows_only": sorted(rows), **out}), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    from paper_2503_24286_gb300 import synth

    rank, world = rank_world()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        BLD.build()
    barrier()
    BLD.build()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = sm_max_mhz_of(local)
    args.fp64_peak = fp64_peak_gflops(n_sm, sm_max)
    path4 = None
    if not args.no_large:
        # the large mechanism's derivative units take minutes to compile: start now
        path4 = large_mechanism_path(synth)
        args.large_compile, large_compile_err = start_large_compile(path4)
    d = tempfile.mkdtemp()
    path = os.path.join(d, "mech.txt")
    synth.write_mechanism(synth.config_mechanism(CONFIG_INDEX), path)
    mech = B.Mechanism(path)
    # compile every kernel group the secondary rows use in one go: NVRTC runs in
    # parallel host threads and the results land in the on-disk cache, which the
    # Crank-Nicolson rows (same mechanism source) hit as well
    groups = [g for g, off in (("jvp,vjp,jacobian", args.no_derivatives), ("jacobian_adiabatic,cn", args.no_cn),
                               ("transport", args.no_transport)) if not off]
    if groups:
        mech.prepare(",".join(groups))
    n = args.points
    cfgd = synth.CONFIGS[CONFIG_INDEX]
    T0, p, Y = synth.generate_states_torch(53, n, cfgd["T"], cfgd["p_atm"],
                                           synth.STATE_SEED_BASE + CONFIG_INDEX + 7919 * rank, dev)
    rho = mech.density(p, T0, Y)
    e = mech.internal_energy(T0, Y)
    del p
    omega = torch.empty((53, n), dtype=torch.float64, device=dev)
    T = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        mech.net_production_rates(rho, Y, e=e, T_out=T, out=omega)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    assert mech.nonconverged() == 0
    # Newton statistics of this batch (not timed)
    _, iters = mech.temperature(e, Y, with_iters=True)
    iters_mean = float(iters.double().mean().item())

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    launches = args.steps          # one fused kernel launch per step
    value = world * n / (ms_max * 1e-3)

    # --- end to end through the C ABI with host buffers (pinned) -------------------
    h_rho = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h_e = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h_Y = torch.empty((53, n), dtype=torch.float64, pin_memory=True)
    h_rho.copy_(rho); h_e.copy_(e); h_Y.copy_(Y)
    h_T = torch.empty(n, dtype=torch.float64, pin_memory=True)
    h_w = torch.empty((53, n), dtype=torch.float64, pin_memory=True)
    a_rho, a_e, a_Y, a_T, a_w = (x.numpy() for x in (h_rho, h_e, h_Y, h_T, h_w))
    h_T.zero_(); h_w.zero_()                      # every output page touched before timing
    # each call is synchronous (host in, host out); its wall time is the step
    e2e_calls = max(10, args.steps)
    for _ in range(2):
        mech.net_production_rates(a_rho, a_Y, e=a_e, T_out=a_T, out=a_w)
    barrier()
    e2e_times = []
    for _ in range(e2e_calls):
        t0 = time.perf_counter()
        mech.net_production_rates(a_rho, a_Y, e=a_e, T_out=a_T, out=a_w)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.median(e2e_times), dev)
    e2e_min_s = max_over_ranks(min(e2e_times), dev)
    h2d = (n + n + 53 * n) * 8
    d2h = (53 * n + n) * 8

    # --- derivative kernels on the 2^20-state workload (JVP, VJP, dense Jacobian) ----------
    deriv = None
    if not args.no_derivatives:
        deriv = derivative_rates(mech, synth, dev, stream, args, rank)
    learned = None
    if not args.no_learned:
        learned = learned_guess_rates(mech, path, synth, dev, stream, args, rank)
    warp53 = None
    large = None
    if not args.no_large:
        mw = B.Mechanism(path, "variant=warp")
        for _ in range(3):
            mw.net_production_rates(rho, Y, e=e, T_out=T, out=omega)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            mw.net_production_rates(rho, Y, e=e, T_out=T, out=omega)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_w = max_over_ranks(e0.elapsed_time(e1) / 3, dev)
        warp53 = {"ms": ms_w, "states_per_s": n / (ms_w * 1e-3)}
        large = large_mechanism_rates(path4, synth, dev, stream, args, rank)
        if large_compile_err:
            large["compile_error"] = large_compile_err[0]
        if args.large_derivatives:
            large["jacobian_type"] = large_derivative_rates(path4, synth, dev, stream, args, rank)

    pdep = None
    if not args.no_pdep:
        pdep = pressure_dependent_rates(synth, dev, stream, args, rank)
    transport = None
    if not args.no_transport:
        transport = transport_rates(mech, synth, dev, stream, args, rank)
    cn = None
    if not args.no_cn:
        cn = crank_nicolson_rates(synth, dev, stream, args, rank)

    # --- roofline of the timed kernel ---------------------------------------------------
    flops_fwd = mech.stat("omega_fp64_flops_per_point")
    flops_ts = 2 * mech.stat("tsolve_collapse_fp64_ops") + 3 * 2 * mech.stat("tsolve_iter_fp64_ops_mixed")
    flops_pt = flops_fwd + flops_ts
    achieved = flops_pt * n / (ms * 1e-3) / 1e9
    src_hash = hashlib.sha256(mech.source().encode()).hexdigest()[:16]
    traffic = PROFILED_TRAFFIC.get(src_hash)
    clocks = clk.summary()

    line = None
    if rank == 0:
        rate_cpu, cores, dt = cpu_oracle_rate(path, args.cpu_sample)
        n1 = max(256, min(args.cpu_sample // 128, 8192))
        rate_1, dt_1 = cpu_oracle_rate_one_core(path, n1)
        line = {"metric": METRIC, "value": value, "unit": "states/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(n),
                "parallelism": "points sharded across ranks, no collective" if world > 1 else "1 GPU",
                "roofline": {"bound": "alu", "achieved": achieved, "peak": args.fp64_peak, "unit": "GFLOP/s",
                             "frac": achieved / args.fp64_peak, "traffic": traffic,
                             "peak_source": "FP64 pipe: 2 lanes/SM/clk (DFMA microbenchmark) x %d SMs (device) x "
                                            "%.0f MHz (nvidia-smi clocks.max.sm) x 2 flops/DFMA" % (n_sm, sm_max),
                             "flops_per_state": flops_pt,
                             "frac_at_sampled_clock": (achieved / (args.fp64_peak * clocks["sm_mhz"] / sm_max)
                                                       if clocks.get("sm_mhz") else None)},
                "cpu_baseline": {"value": rate_cpu, "unit": "states/s", "cores": cores, "kind": "oracle",
                                 "sample": "%d states of the same workload (seeded), T solve + omega, %.1f s"
                                           % (args.cpu_sample, dt),
                                 "value_one_core": rate_1,
                                 "sample_one_core": "%d states, 1 thread, %.1f s" % (n1, dt_1)},
                "e2e": {"value": world * n / e2e_s, "unit": "states/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "calls": e2e_calls, "statistic": "median call",
                        "value_best_call": world * n / e2e_min_s},
                "gpu_launches": launches,
                "clocks": clocks,
                "newton_iters_mean": iters_mean,
                "jacobian_evals_per_s": deriv["jacobian_per_s"] if deriv else None,
                "derivatives": deriv,
                "learned_guess": learned,
                "warp_per_state_53sp": warp53,
                "large_mechanism": large,
                "crank_nicolson": cn,
                "transport": transport,
                "pressure_dependent": pdep,
                "kernel_source_hash": src_hash,
                "kernel": "pyro_omega (fused Newton T(e,Y) + omega), %d threads/block, %d blocks/SM"
                          % (int(mech.stat("block")), int(mech.stat("omega_blocks_per_sm")))}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--points", type=int, default=2 ** 22)
    ap.add_argument("--cpu-sample", type=int, default=2 ** 20)
    ap.add_argument("--ref-sample", type=int, default=2 ** 15)
    ap.add_argument("--deriv-points", type=int, default=2 ** 20)
    ap.add_argument("--no-derivatives", action="store_true")
    ap.add_argument("--train-points", type=int, default=2 ** 24)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--large-points", type=int, default=2 ** 21)
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--large-derivatives", nargs="?", const="jacobian,jacobian_adiabatic,cn", default=None,
                    help="also time the Jacobian, dS/dY and Crank-Nicolson kernels on the 160-species "
                         "mechanism (or the comma list given of jacobian, jacobian_adiabatic, cn)")
    ap.add_argument("--large-deriv-points", type=int, default=2 ** 15)
    ap.add_argument("--large-jac-points", type=int, default=2 ** 15,
                    help="states of the block-per-state dense Jacobian rows of the large mechanism")
    ap.add_argument("--cn-points", type=int, default=2 ** 18)
    ap.add_argument("--no-cn", action="store_true")
    ap.add_argument("--transport-points", type=int, default=2 ** 20)
    ap.add_argument("--no-transport", action="store_true")
    ap.add_argument("--pdep-points", type=int, default=2 ** 22)
    ap.add_argument("--no-pdep", action="store_true")
    ap.add_argument("--only", default=None,
                    help="profiling: run only these secondary rows (comma list of derivatives, learned, large, pdep, "
                         "transport, cn) and print them; no headline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        rc = run_reference(args)
    else:
        rc = run_rows_only(args) if args.only else run_ours(args)
    dist = _dist()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
