"""Benchmark: damped real Chebyshev steps/s on the J = 10 H + DH workload.

Workload: 256 (R) x 192 (r) x 96 (gamma) grid, J = 10 with helicities 0..10
(11 Coriolis-coupled blocks, 51.9 M grid values), synthetic Sato LEPS surface,
500 energies in the flux sums, reactant-channel projections (v <= 3, j <= 15).
One step = one full Chebyshev iteration of the hot path: radial kinetic
transforms, gamma transforms with FBR/Coriolis, potential, damped recursion,
flux cut, channel overlaps, norms, plus the amortised energy-sum GEMM.

value: steps/s of the mixed form (FP32 state, FP64 energy sums), inputs resident
in HBM. The FP64 form is measured too ("fp64"). e2e: the same step through the
public C ABI with host buffers (state uploaded, probabilities read back, each
step). --impl reference times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

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

WORKLOAD = "h_dh_j10_256x192x96_11omega"
# the headline is config 2; --config times another workload with the same line
WORKLOADS = {"c2": WORKLOAD, "c3": "two_state_j0to30_192x128x64_164blocks",
             "c4": "h_dh_j40_512x384x180_21omega"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # defaults: whole energy rings (128 iterations each), the first ring's CUDA graph captured
    # during the warm-up, and a timed region long enough for several clock samples
    ap.add_argument("--steps", type=int, default=1280)
    ap.add_argument("--warmup", type=int, default=256)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=3)
    # accuracy gate of the headline: mixed against the FP64 GPU path from the initial packet
    # (0 skips it; the configured length of the workload is 12000 iterations)
    ap.add_argument("--accuracy-steps", type=int, default=None,
                    help="default 1280 for config 2, 0 (skipped) for the others")
    ap.add_argument("--config", default="c2", choices=sorted(WORKLOADS),
                    help="workload (config 2 is the headline; config 3 and 4 are timed the "
                         "same way, without the CPU baseline unless --cpu-baseline)")
    ap.add_argument("--cpu-baseline", action="store_true")
    ap.add_argument("--no-pcb", action="store_true",
                    help="skip the products-coordinate start timing (config 2's product grid)")
    a = ap.parse_args()
    if a.accuracy_steps is None:
        a.accuracy_steps = 1280 if a.config == "c2" else 0
    if a.config != "c2" and not a.cpu_baseline:
        a.no_cpu_baseline = True
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_oracle_rate(nsteps):
    """Times the FP64 oracle (as it stands) for nsteps Chebyshev iterations of the
    workload in a child process on all host cores; returns (steps/s, cores, seconds)."""
    cores = os.cpu_count() or 1
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import workloads as W\n"
        "from oracle import propagate as P\n"
        "from oracle.hamiltonian import GridHamiltonian\n"
        "cfg = W.C2\n"
        "H = GridHamiltonian(cfg)\n"
        "t = time.perf_counter(); P.propagate(cfg, nsteps=%d, H=H)\n"
        "dt = time.perf_counter() - t\n"
        "t2 = time.perf_counter(); P.propagate(cfg, nsteps=0, H=H); d0 = time.perf_counter() - t2\n"
        "print(json.dumps({'dt': dt, 'setup': d0}))\n" % (ROOT, nsteps))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    per = max(d["dt"] - d["setup"], 1e-9)   # per-propagation setup (channels, packet) excluded
    return nsteps / per, cores, per


# ----------------------------------------------------------- reference arm
REF_MAX_STEPS = 8


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import workloads as W
    cfg = W.C2
    npts = cfg["grid"]["NR"] * cfg["grid"]["nr"] * cfg["grid"]["ngamma"] * 11
    # each step: one full oracle Chebyshev iteration of the workload (about 5 s on 16 cores);
    # the timed sample is capped at REF_MAX_STEPS iterations (and one warm-up iteration) so
    # that the run ends within about a minute whatever --steps asks for
    n_warm = min(args.warmup, 1)
    n_timed = max(1, min(args.steps, REF_MAX_STEPS))
    if n_warm > 0:
        cpu_oracle_rate(n_warm)
    rate, cores, secs = cpu_oracle_rate(n_timed)
    line = {
        "impl": "reference", "metric": "Chebyshev steps/s", "value": rate, "unit": "steps/s",
        "n_gpus": 0, "steps": n_timed, "warmup": n_warm, "ms_per_step": 1e3 / rate,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Sato LEPS H+DH)",
        "config": {"workload": WORKLOAD, "grid_pts_omega": npts, "energies": 500},
        "grid_pts_omega_per_s": rate * npts,
        "cpu_baseline": {"value": rate, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{n_timed} oracle iterations of the full workload "
                                   f"({secs:.1f} s; --steps {args.steps} capped at {REF_MAX_STEPS})"},
        "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- our arm
def captured_traffic(kernel_key):
    """DRAM bytes per launch of `kernel_key` from the committed ncu capture record
    (profiles/traffic_<kernel_key>_c2_mixed.txt), or None when the kernel's source file has
    changed since the capture (its SHA-1 is part of the record)."""
    import hashlib
    rec = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                       f"traffic_{kernel_key}_c2_mixed.txt")
    try:
        fields = {}
        with open(rec) as f:
            for ln in f:
                if ln.strip() and not ln.startswith("#"):
                    k, _, v = ln.strip().partition(" ")
                    fields[k] = v.strip()
        src = os.path.join(os.path.dirname(os.path.abspath(__file__)), fields["source"])
        with open(src, "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != fields["source_sha1"]:
                return None
        return float(fields["dram_bytes"])
    except (OSError, KeyError, ValueError):
        return None


def kernel_roofline(kernel, es, npts, nblk, ng, nelec, nE, kb, ncols):
    """Algorithmic work of one launch of `kernel` on the workload: (bound, amount).

    bound "hbm": bytes the launch must move at minimum; "alu": FLOPs (CUDA cores).
    vec = one state vector (nblk * npts values of es bytes)."""
    vec = npts * nblk * es
    if kernel == "kinetic_rows":
        return "hbm", 2 * vec                   # read c_k, write t
    if kernel == "kinetic_cols":
        return "hbm", 3 * vec                   # read c_k, read + write t
    if kernel == "kinetic_radial":
        return "hbm", 2 * vec                   # read c_k, write t (both radial terms)
    if kernel == "gamma_to_dvr":
        return "alu", 2.0 * ng * ng * (npts // ng) * nblk
    if kernel == "gamma_update":
        return "alu", 2.0 * ng * ng * (npts // ng) * nblk
    if kernel == "norms":
        return "hbm", vec                       # read c_(k+1)
    if kernel == "sums_flush":
        return "alu", 2.0 * (2 * nE) * kb * ncols
    if kernel == "channels":
        return "hbm", es * nblk * ng * 0 + 8
    if kernel == "angular_tc":
        # the method's own minimum per step (read q_k, read q_(k-1), write q_(k+1)) plus the
        # potential of the J (shared by its Omega blocks); the unfused design also reads t
        return "hbm", 3 * vec + (npts * es) * nelec * nelec
    return "hbm", vec


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import workloads as W
    from paper_2412_10167_gb300 import mw3

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    cfg = W.CONFIGS[args.config]
    g = cfg["grid"]
    nelec = cfg["nelec"]
    nblk = sum(min(J, cfg["omega_max"]) + 1 for J in cfg["J"]) * nelec
    nE = cfg["analysis"]["nE"]
    npts = g["NR"] * g["nr"] * g["ngamma"]

    from paper_2412_10167_gb300 import dist as mdist

    def barrier():
        mdist.barrier()
        torch.cuda.synchronize()

    # ---- mixed form: the headline
    pr = mw3.Propagator(cfg, device=local, precision="mixed")
    pr.propagate(args.warmup)
    kb = pr.get_tuning("kb")
    clk = ClockSampler(local)
    # CUDA events on the library's stream (the stream its kernels are launched on)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    clk.start()
    ev0.record(pr.stream)
    pr.propagate(args.steps)
    ev1.record(pr.stream)
    barrier()
    clocks = clk.stop()
    elapsed = mdist.max_over_ranks(ev0.elapsed_time(ev1) * 1e-3)
    value = world * args.steps / elapsed
    # per-kernel CUDA-event times: a second pass of the same length with the library's kernel
    # timers on. They record events around every launch, which keeps full chunks out of CUDA
    # graphs, so the headline pass above runs without them.
    pr.kernel_times(enable=True)
    pr.propagate(args.steps)
    ktimes = pr.kernel_times()
    pr.kernel_times(enable=False)
    nchan = 0
    E, Pmix, _ = pr.probabilities()

    # ---- e2e through the public API with host buffers
    q_dev, qp_dev = pr.state()
    # the step's inputs sit in pinned (page-locked) host memory, FP32 like the mixed form's
    # state (mw3_set_state_f32)
    q_host = torch.empty(q_dev.shape, dtype=torch.float32, pin_memory=True).numpy()
    qp_host = torch.empty(qp_dev.shape, dtype=torch.float32, pin_memory=True).numpy()
    q_host[...] = q_dev
    qp_host[...] = qp_dev
    # two whole cycles of pending energy-ring reads (the mixed form adds up to sixteen pending
    # iterations on the fly; the seventeenth read flushes)
    e2e_steps = max(4, min(34, args.steps // 8))
    # one untimed iteration: upload buffers, the copy stream and the cached packet amplitudes
    # are set up on first use
    pr.set_state_f32(q_host, qp_host)
    pr.propagate(1)
    pr.probabilities()
    barrier()
    te0 = time.perf_counter()
    tparts = [0.0, 0.0, 0.0]   # host wall time of the three calls (each returns synchronised)
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        pr.set_state_f32(q_host, qp_host)
        t1 = time.perf_counter()
        pr.propagate(1)
        t2 = time.perf_counter()
        _, Pe, _ = pr.probabilities()
        t3 = time.perf_counter()
        tparts[0] += t1 - t0
        tparts[1] += t2 - t1
        tparts[2] += t3 - t2
    barrier()
    te = mdist.max_over_ranks(time.perf_counter() - te0)   # wall clock: host copies included
    prod_launches = 3 if pr.get_tuning("prod_gather") else 2
    pr.close()
    del pr

    # ---- FP64 form on the same workload (shorter timed region)
    pf = mw3.Propagator(cfg, device=local, precision="fp64")
    pf.propagate(max(3, min(args.warmup, 8)))
    fe0 = torch.cuda.Event(enable_timing=True)
    fe1 = torch.cuda.Event(enable_timing=True)
    barrier()
    fe0.record(pf.stream)
    pf.propagate(args.fp64_steps)
    fe1.record(pf.stream)
    barrier()
    tf = mdist.max_over_ranks(fe0.elapsed_time(fe1) * 1e-3)
    fp64_rate = world * args.fp64_steps / tf
    pf.close()
    del pf

    # ---- accuracy of the mixed form: both forms from the initial packet for the same count
    accuracy = None
    if args.accuracy_steps > 0 and rank == 0:
        res = {}
        for prec in ("mixed", "fp64"):
            pa = mw3.Propagator(cfg, device=local, precision=prec)
            pa.propagate(args.accuracy_steps)
            _, Pt_, Pin_ = pa.probabilities()
            res[prec] = (Pt_, Pin_, pa.product_probabilities(), pa.norm_trace()[-1][0])
            pa.close()
            del pa
        (mt, mi, mp, _), (ft, fi, fp_, fnorm) = res["mixed"], res["fp64"]
        d = {"total": float(np.max(np.abs(mt - ft))),
             "reactant_channels": float(np.max(np.abs(mi - fi))),
             "product_channels": float(np.max(np.abs(mp - fp_)))}
        accuracy = {
            "iterations": args.accuracy_steps,
            "against": "FP64 GPU path (equal to the FP64 oracle to 1e-8 in the parity tests)",
            "max_abs_dP": d, "gate": 1e-4, "pass": max(d.values()) <= 1e-4,
            "fp64_range": {"P_total": [float(ft.min()), float(ft.max())],
                           "reactant_channel_sum_max": float(fi.sum(axis=(1, 2, 3)).max()),
                           "product_channel_sum_max": float(fp_.sum(axis=(1, 2, 3)).max())},
            "fp64_final_norm": float(fnorm),
        }

    # ---- products-coordinate-based start: the one-off carry of the H + DH packet onto the
    # product-arrangement grid of the same size class (256 x 256 x 96, J = 10, 11 blocks)
    pcb_start = None
    if rank == 0 and not args.no_pcb and args.config == "c2":
        pcfg = W.PCB["c2pcb"]
        pp = mw3.Propagator(pcfg, device=local, precision="mixed", analysis=False)
        pp.kernel_times(enable=True)
        t0 = time.perf_counter()
        pp.init_packet()
        t_call = time.perf_counter() - t0
        kms, kn = pp.kernel_times()["pcb_packet"]
        pp.kernel_times(enable=False)
        q_p, _ = pp.state()
        pg = pcfg["grid"]
        pnodes = pg["NR"] * pg["nr"] * pg["ngamma"]
        pblk = sum(min(J, pcfg["omega_max"]) + 1 for J in pcfg["J"]) * pcfg["nelec"]
        pcb_start = {"workload": pcfg["name"], "kernel_ms": kms / max(kn, 1),
                     "call_ms": 1e3 * t_call, "nodes": pnodes, "blocks": pblk,
                     "node_blocks_per_s": pnodes * pblk / (1e-3 * kms / max(kn, 1)),
                     "carried_norm": float(np.sum(q_p.astype(np.float64) ** 2))}
        pp.close()
        del pp

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    per = {k: (ms / n if n else 0.0, n) for k, (ms, n) in ktimes.items()}
    dom = max((k for k in per if per[k][1] > 0), key=lambda k: per[k][0] * per[k][1])
    avg_ms = per[dom][0]
    es = 4
    fp32_peak = fp64_peak = None
    try:
        fp32_peak = mw3.mw3_measure_peak(local, 1)
        fp64_peak = mw3.mw3_measure_peak(local, 0)
    except Exception:
        pass
    ncols_total = 2 * nblk * g["ngamma"] * g["NR"]   # the flux-cut columns of the ring
    bound, amount = kernel_roofline(dom, es, npts, nblk, g["ngamma"], nelec, nE, kb,
                                    ncols_total)
    if bound == "alu":
        ach = amount / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (ach / fp32_peak) if fp32_peak else None, "traffic": None, "kernel": dom,
                "peak_source": "measured FP32 FMA-chain probe (mw3_measure_peak)"}
    else:
        ach = amount / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": captured_traffic(dom), "kernel": dom,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    kernels = {k: {"avg_ms": round(per[k][0], 5), "launches": per[k][1],
                   "share": round(per[k][0] * per[k][1] / max(1e-9, sum(a * b for a, b in per.values())), 4)}
               for k in per if per[k][1]}
    # kernels per timed launch group on the tensor-core mixed path: the angular step is the
    # tcgen05 kernel and the norm reduction, products are the node and dot kernels, a flush is
    # the phase table and the ring GEMM; the others are one kernel each
    # (three for the products in the plane-major form: the column gather, the node sums and
    # the dots)
    per_group = {"angular_tc": 2, "products": prod_launches, "sums_flush": 2}
    launches = sum(v[1] * per_group.get(k, 1) for k, v in per.items())

    cpu = None
    if not args.no_cpu_baseline:
        try:
            rate, cores, secs = cpu_oracle_rate(args.cpu_sample_steps)
            cpu = {"value": rate, "unit": "steps/s", "cores": cores, "kind": "oracle",
                   "cpu_model": cpu_model(),
                   "sample": f"{args.cpu_sample_steps} FP64 oracle iterations of the full workload "
                             f"({secs:.1f} s)"}
        except Exception as e:  # report, do not hide
            cpu = {"value": None, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {str(e)[:200]}"}

    vec_bytes = nblk * npts * 4   # FP32 host state of the e2e arm
    line = {
        "metric": "Chebyshev steps/s", "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64sums",
        "data": "synthetic (Sato LEPS H+DH surface, deterministic packet)",
        "config": {"workload": WORKLOADS[args.config], "grid": [g["NR"], g["nr"], g["ngamma"]],
                   "J": cfg["J"] if len(cfg["J"]) > 1 else cfg["J"][0], "electronic_states": nelec,
                   "blocks": nblk, "energies": nE, "kb": kb,
                   # energy rings that fill inside the timed region are flushed there; slots
                   # of a ring still open at its end stay pending (a probability read adds
                   # them), so K not a multiple of kb leaves that share of a flush untimed
                   "flushes_timed": (args.warmup + args.steps) // kb - args.warmup // kb,
                   "ring_slots_pending_after": (args.warmup + args.steps) % kb,
                   "l2": f"state vectors {nblk * npts * 4 / 1e6:.0f} MB each (> 129 MB L2), "
                         "no flush needed",
                   "parallelism": f"replicas x{world}"},
        "grid_pts_omega_per_s": value * npts * nblk,
        "fp64": {"value": fp64_rate, "unit": "steps/s", "steps": args.fp64_steps,
                 "grid_pts_omega_per_s": fp64_rate * npts * nblk},
        "mixed_over_fp64": value / fp64_rate,
        "roofline": roof,
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": world * e2e_steps / te, "unit": "steps/s",
                # the two state vectors up, and the |a(E)|^2 row of the probability read
                "h2d_bytes_per_step": 2 * vec_bytes + nE * 8,
                # back: the flux per (J, E) and the channel probabilities per (J, Lambda, v, j, E)
                "d2h_bytes_per_step": 8 * len(cfg["J"]) * nE * (1 + nelec * (cfg["analysis"]["vmax"] + 1)
                                                                * (cfg["analysis"]["jmax"] + 1)),
                "host_state": "f32 pinned",
                "steps": e2e_steps,
                "ms_per_call": {"set_state_f32": 1e3 * tparts[0] / e2e_steps,
                                "propagate_1": 1e3 * tparts[1] / e2e_steps,
                                "probabilities": 1e3 * tparts[2] / e2e_steps}},
        "accuracy": accuracy,
        "cpu_baseline": cpu,
        "fp32_fma_peak_tflops": fp32_peak,
        "fp64_fma_peak_tflops": fp64_peak,
        "pcb_start": pcb_start,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
