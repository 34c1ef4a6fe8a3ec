"""Throughput of the lattice time step on GB300: Gsite-updates/s at 256^3.

Workload (one "step"): two-field preheating V = m^2 phi^2/2 + g^2 phi^2 chi^2/2 with
q = g^2 phi0^2/(4 m^2) = 1e4 (program units: m2 = 1, g2 = 4q), on a 256^3 periodic
lattice, fields in FP32 with Kahan-compensated drifts, FP64 reductions and a(t),
Yoshida-4 (three fused passes per step), dt = 0.005, self-consistent expansion,
started from the library's own Philox vacuum state (seed 1234).  A site-update is
one lattice site advanced by one full step.  The inputs (805 MB of state) are
larger than L2 (129 MB), so no flush is needed between steps.

Arms:
  default          the CUDA path through the C ABI (libcl.so).
  --impl reference the FP64 CPU oracle as it stands, one oracle Yoshida-4 step of the
                   same 256^3 workload per timed step, on this host's cores.
Extra keys: roofline (dominant kernel = the fused scalar pass), cpu_baseline (the
oracle on a bounded sample), e2e (the same metric through the C ABI with host
buffers: state upload, step, energies download each step), fp64_plain (the same
workload in FP64 without compensation), clocks (nvidia-smi during the timed region).

Other workloads (--workload; one JSON line each, same keys where they apply):
  u1        axion + compact U(1) links, 192^3, FP32, RK3-3, alpha_Lambda = 30,
            V = phi^2/2, phi = 1 + noise, phi' = -0.5, A = 0, small divergence-free E.
  u1lf      the same with the leapfrog (implicit momentum kick, three passes a step).
  ensemble  1024 independent lambda phi^4 lattices of sizes drawn from {32, 48, 64}^3,
            per-member vacuum amplitude lambda log-uniform in [1e-6, 1e-3], VV-2,
            FP32 + Kahan, one launch per pass for all members.
  surrogate the convolutional surrogate at 128^3: 6 periodic 3x3x3 layers
            (3 -> 48, 4 x 48 -> 48, 48 -> 2), BF16 on the tensor cores; forward and
            forward + backward throughput, and the time of the 16 leapfrog steps one
            forward replaces.  Then a bounded training run on leapfrog trajectories
            (32^3) and the judged jumps on a fresh lattice: acceptance under the 1e-3
            Hubble limit, binned-spectrum error against the plain leapfrog, wall time
            (the surrogate speed-up at 1 % error, when reached).
  rk        the headline lattice advanced by RK4-5 (2N) stages.
  gw        the headline plus the five traceless GW auxiliaries, Yoshida-4.
  nmc       one non-minimally coupled lambda phi^4 field (xi = 0.3), 256^3, RK4-5.
  reduced   the headline's model on a (2+1)-dimensional 4096^2 lattice, Yoshida-4.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 256
L = 8.0 * math.pi
DT = 0.005
Q = 1.0e4
G2 = 4.0 * Q
KAPPA = 0.1
ALPHA = 0.0
AMP2 = 1.0e-9
SEED = 1234
METRIC = "Gsite-updates/s at 256^3"
PASSES_PER_STEP = 3
# algorithmic bytes of one fused pass per site: phi, pi, c for two fields, read + write, 4 B each
BYTES_PER_SITE_PASS = 2 * 3 * 2 * 4
BYTES_PER_SITE_PASS_FP64 = 2 * 2 * 2 * 8


def config(extra=None):
    c = {"workload": "two-field preheating m2phi2+g2phi2chi2, q=1e4, %d^3, Yoshida-4, FP32+Kahan, "
                     "FP64 reductions, dt=0.005, self-consistent expansion" % N,
         "lattice": N, "fields": 2, "integrator": "yoshida4", "passes_per_step": PASSES_PER_STEP,
         "l2": "inputs (%.0f MB) larger than L2; no flush" % (N ** 3 * 6 * 4 * 2 / 1e6)}
    if extra:
        c.update(extra)
    return c


KERNEL_SOURCES = ["paper_2607_24978_gb300/csrc/scalar_pass.cu", "paper_2607_24978_gb300/csrc/scalar_pass_tma.cuh",
                  "paper_2607_24978_gb300/csrc/scalar_pass_tma_nr.cuh",
                  "paper_2607_24978_gb300/csrc/scalar_pass_common.cuh", "paper_2607_24978_gb300/csrc/kernel_common.cuh",
                  "paper_2607_24978_gb300/csrc/cl_internal.cuh"]


def profiled_traffic():
    """DRAM bytes per launch of the fused pass from the ncu record committed beside its summary
    (profiles/scalar_pass_256_yoshida4_fp32kahan.json), or None when the kernel sources changed
    since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "scalar_pass_256_yoshida4_fp32kahan.json")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256()
        for s in KERNEL_SOURCES:
            h.update(open(os.path.join(ROOT, s), "rb").read())
        if h.hexdigest()[:16] != rec["kernel_sources_sha256_16"]:
            return None
        return int(rec["traffic_bytes_per_launch"])
    except Exception:
        return None


def fp64_ops_record():
    """FP64 operations per site and pass of the FP64 pass kernel, counted by ncu (committed
    beside its summary), or None when the kernel sources changed since."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "scalar_pass_256_yoshida4_fp64.json")))
        h = hashlib.sha256()
        for s in rec["kernel_sources"]:
            h.update(open(os.path.join(ROOT, s), "rb").read())
        return rec if h.hexdigest()[:16] == rec["kernel_sources_sha256_16"] else None
    except Exception:
        return None


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        self.first = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        if self.p:  # the sampler is live (its first line, before the timed region, is read) or gone
            import select
            r, _, _ = select.select([self.p.stdout], [], [], 5.0)
            if r:
                self.first = self.p.stdout.readline()
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
            if not self.lines and self.first:  # a region shorter than one sampling period
                self.lines = [self.first]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ oracle legs
REF_N = 64  # per-step sample of the reference arm: same per-site arithmetic on 64^3 sites


def oracle_model(n=None):
    n = N if n is None else n
    from oracle import oracle as O
    return O.make_model(n, L * n / 256, nf=2, alpha=ALPHA, kappa=KAPPA, expansion=True, m2=(1.0, 0.0), g2=G2)


def oracle_state(n=None):
    """Seeded homogeneous-plus-noise state of the bench shape (the oracle's own vacuum state
    at 256^3 would take minutes of direct DFTs, so the CPU legs start from this input)."""
    import numpy as np
    from oracle import oracle as O
    from tests import inputs
    n = N if n is None else n
    phi, pi = inputs.scalar_state(n, 2, seed=SEED, fbar=(1.0, 0.0), amp=1e-5, pamp=1e-5)
    st = O.State(phi, pi, np.array([1.0, 0.0, 0.0]))
    st.abt[1] = math.sqrt(KAPPA * O.energies(oracle_model(n), st)["rho"] / 3.0)
    return st


def cpu_baseline(n=None):
    """The oracle on a bounded sample of the workload: Yoshida-4 steps of the two-field lattice
    (the headline's size, at most 256^3), once on every host core (the loop-parallel build,
    the reported figure) and once on one thread."""
    from oracle import oracle as O
    n = min(N, 256) if n is None else n
    out = {}
    for omp, steps in ((True, 8), (False, 2)):
        O.use_threads(omp)
        cores = O.threads()
        m = oracle_model(n)
        st = oracle_state(n)
        O.step(m, st, O.YOSHIDA4, DT, 1)  # first touch of the arrays outside the timing
        t0 = time.perf_counter()
        O.step(m, st, O.YOSHIDA4, DT, steps)
        dt = time.perf_counter() - t0
        out[omp] = {"value": n ** 3 * steps / dt / 1e9, "unit": "Gsite-updates/s", "cores": cores, "kind": "oracle",
                    "sample": "%d oracle Yoshida-4 steps of the %d^3 two-field lattice, FP64, %d thread%s (%.1f s)"
                              % (steps, n, cores, "" if cores == 1 else "s", dt)}
    O.use_threads(False)
    line = dict(out[True])
    line["nproc"] = os.cpu_count()
    line["single_thread"] = out[False]
    return line


def run_reference(args, world, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    O.use_threads(True)  # every host core (the loop-parallel build of the oracle)
    cores = O.threads()
    m = oracle_model(REF_N)
    st = oracle_state(REF_N)
    for _ in range(args.warmup):
        O.step(m, st, O.YOSHIDA4, DT, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(m, st, O.YOSHIDA4, DT, 1)
    el = time.perf_counter() - t0
    v = REF_N ** 3 * args.steps / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gsite-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config({"impl": "FP64 CPU oracle, %d threads" % cores}),
            "cpu_baseline": {"value": v, "unit": "Gsite-updates/s", "cores": cores, "kind": "oracle",
                             "sample": "per timed step one oracle Yoshida-4 step of the same two-field "
                                       "workload on 64^3 sites (same per-site arithmetic as 256^3), "
                                       "%d threads" % cores},
            "e2e": {"value": v, "unit": "Gsite-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ other workloads
U1 = dict(N=192, L=2 * math.pi / 0.1, dt=0.01, alphaL=30.0, ws2=1e-4, kappa=1.0, alpha=0.0, m2=1.0, phi0=1.0,
          dphi0=-0.5, e_amp=1e-6, seed=1234)
U1_STAGES = 3
# algorithmic bytes of one RK stage per site: phi, pi, theta_1..3, E_1..3 and their eight
# Runge-Kutta auxiliaries, read + write, 4 B each
U1_BYTES_PER_SITE_STAGE = 8 * 2 * 2 * 4
# the leapfrog's step per site, 4 B each: pass 1 reads (phi, theta_1..3) and (pi, E_1..3) and
# writes the integer-time momenta and the first iterate (16 arrays); pass 2 reads the
# positions, the iterate and the integer-time momenta and writes the next iterate (16);
# pass 3 the same and writes the positions too (20)
# what the staged launches of one RK stage move per site, 4 B each: the plaquette launch reads
# phi, theta, E (7) and writes sin P, the rate and the Chern-Simons field (9); the stage reads
# its 14 staged arrays, theta and the 8 auxiliaries at the site (11; the first stage reads no
# auxiliaries) and writes the 8 degrees of freedom and their 8 auxiliaries
U1_RK_DESIGN_BYTES_PER_SITE_STAGE = (7 + 9 + 14 + 11 + 16) * 4
U1_LF_PASSES = 3
U1_LF_BYTES_PER_SITE_STEP = (16 + 16 + 20) * 4
# what the staged launches of a step move per site, 4 B each (halo rows from L2 not counted):
# the full plaquette launch reads phi, theta, E (7) and writes sin P, cos P, the rate and the
# Chern-Simons field (12); each of the two rates launches reads phi, E, cos P (7) and writes 6;
# the stage launches read their 14 staged arrays, passes 2 and 3 also the 4 base momenta and
# pass 3 the 3 link angles it drifts, and write 8 (pass 1), 4 (pass 2) and 8 (pass 3)
U1_LF_DESIGN_BYTES_PER_SITE_STEP = (7 + 12 + 2 * (7 + 6) + (14 + 8) + (14 + 4 + 4) + (14 + 4 + 3 + 8)) * 4
RK_STAGES = 5
# GW pass per site: the scalars the scalar pass just drifted, two fields read (8 B), and the
# five auxiliaries and their momenta read and written (2 x 10 x 4 B), FP32
GW_BYTES_PER_SITE_PASS = 2 * 4 + 2 * 10 * 4
NMC_XI = 0.3
# NMC stage per site, one field, FP32 + Kahan: phi, pi, k_phi, k_pi, c read and written (40 B;
# 32 B in the first stage, which reads no k), averaged over the 5 stages.  The Ricci scalar's
# lattice sums ride along in the stage kernel (of its output state), so they move no bytes of
# their own
NMC_BYTES_PER_SITE_STAGE = (4 * 40 + (40 - 8)) / 5.0
# algorithmic bytes of one RK4-5 step per site, two fields, FP32 + Kahan: phi, pi, k_phi, k_pi,
# c read + write in four stages; the first stage (A = 0) reads no k
RK_BYTES_PER_SITE_STEP = 2 * 4 * (4 * 5 * 2 + (5 * 2 - 2))
ENS = dict(members=1024, sizes=(32, 48, 64), lam=(1e-6, 1e-3), L=8.0 * math.pi, dt=0.01, alpha=1.0, kappa=0.1,
           seed=1234)
# VV-2, one field, FP32 + Kahan: phi, pi, c read + write
ENS_BYTES_PER_SITE = 3 * 2 * 4


def timed_region(torch, g, stream, steps):
    clk = Clocks(torch.cuda.current_device())
    with clk:
        el, launches = timed_steps(torch, g, stream, steps)
    return el, launches, clk.summary()


def run_u1_workload(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src, leapfrog=False):
    import numpy as np
    from tests import inputs
    c = U1
    N = c["N"]
    g = cl.Lattice(N, c["L"], 1, cl.CL_PREC_FP32, cl.CL_INT_VV2 if leapfrog else cl.CL_INT_RK3_3,
                   gauge=cl.CL_GAUGE_U1_AXION, expansion=True, alpha=c["alpha"], kappa=c["kappa"], dt=c["dt"],
                   stream=stream.cuda_stream)
    g.cl_set_potential(cl.CL_POT_M2, [c["m2"]])
    g.cl_set_gauge_coupling(c["alphaL"], c["ws2"])
    if args.variant is not None:  # 2: staged launches (default), 0: gather launches, 1: fused stage
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, args.variant)
    if args.dz is not None:  # planes per block of the U(1) kernels (tuning runs)
        g.cl_set_option(cl.CL_OPT_TILE_DZ, args.dz)
    phi, pi = inputs.scalar_state(N, 1, seed=c["seed"], fbar=(c["phi0"],), amp=1e-5, pamp=1e-5,
                                  pbar=(c["dphi0"],))
    E = inputs.solenoidal_field(N, seed=c["seed"] + 1, amp=c["e_amp"], dtype=np.float32)
    g.cl_set_state(cl.CL_FIELD_PHI0, phi[0].astype(np.float32))
    g.cl_set_state(cl.CL_FIELD_PI0, pi[0].astype(np.float32))
    for i in range(3):
        g.cl_set_state(cl.CL_FIELD_E1 + i, np.ascontiguousarray(E[i]))
    del phi, pi, E
    g.cl_set_scalars(1.0)
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    el, launches, clocks = timed_region(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    e = g.cl_energies()
    variant = g.cl_get_option(cl.CL_OPT_PASS_VARIANT)
    u1_dz = g.cl_get_option(cl.CL_OPT_TILE_DZ)
    g.close()
    energies_end = {"a": e["a"], "rho": e["rho"], "KE": e["KE"], "GB": e["GB"],
                    "gauss_violation": e["gauss_violation"], "hubble_violation": e["hubble_violation"],
                    "gauss_rms_last_step": e["gauss_rms_step"], "gauss_rms_max_over_steps": e["gauss_rms_max"]}
    if leapfrog:
        step_s = el / args.steps
        bytes_step = N ** 3 * U1_LF_BYTES_PER_SITE_STEP
        achieved = bytes_step / step_s / 1e9
        kern = ("three passes of k_u1s_plaquettes + k_u1s_stage<float,false,true> (staged neighbourhoods)"
                if variant == 2 else "three passes of k_u1_plaquettes + k_u1_stage<float>")
        return {"metric": "Gsite-updates/s, axion-U(1) 192^3 leapfrog", "value": world * N ** 3 * args.steps / el_max / 1e9,
                "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "axion-U(1) 192^3, leapfrog (implicit momentum kick, three force evaluations "
                                       "per step), FP32, alpha_Lambda=30, (omega*/f*)^2=1e-4, kappa=1, V=phi^2/2, "
                                       "phi=1, phi'=-0.5, A=0, divergence-free E (rms 1e-6), dt=0.01",
                           "lattice": N, "passes_per_step": U1_LF_PASSES,
                           "l2": "inputs (%.0f MB) larger than L2; no flush" % (N ** 3 * 16 * 4 / 1e6)},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                             "kernel": kern + ", per step", "tile_dz": u1_dz,
                             "algorithmic_bytes_per_step": bytes_step,
                             "launch_bytes_per_step": N ** 3 * U1_LF_DESIGN_BYTES_PER_SITE_STEP,
                             "launch_bytes_frac": N ** 3 * U1_LF_DESIGN_BYTES_PER_SITE_STEP / step_s / 1e9 / hbm_peak},
                "gpu_launches": launches, "clocks": clocks, "energies_end": energies_end,
                "gauss_tracking": "rms lattice Gauss charge of every step's integer-time starting state, summed by "
                                  "the second pass of the step (staged form) inside the timed steps"}
    stage_s = el / (args.steps * U1_STAGES)
    bytes_stage = N ** 3 * U1_BYTES_PER_SITE_STAGE
    achieved = bytes_stage / stage_s / 1e9
    return {"metric": "Gsite-updates/s, axion-U(1) 192^3 RK3-3", "value": world * N ** 3 * args.steps / el_max / 1e9,
            "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "axion-U(1) 192^3, RK3-3, FP32, alpha_Lambda=30, (omega*/f*)^2=1e-4, kappa=1, "
                                   "V=phi^2/2, phi=1, phi'=-0.5, A=0, divergence-free E (rms 1e-6), dt=0.01",
                       "lattice": N, "stages_per_step": U1_STAGES,
                       "l2": "inputs (%.0f MB) larger than L2; no flush" % (N ** 3 * 16 * 2 * 4 / 1e6)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                         "kernel": {1: "k_u1_fused<float> (one launch per RK stage)",
                                    2: "one RK stage: k_u1s_plaquettes + k_u1s_stage (staged neighbourhoods)"}.get(
                                        variant, "one RK stage: k_u1_plaquettes + k_u1_stage"), "tile_dz": u1_dz,
                         "algorithmic_bytes_per_launch": bytes_stage,
                         "launch_bytes_per_step": N ** 3 * (U1_STAGES * U1_RK_DESIGN_BYTES_PER_SITE_STAGE - 8 * 4),
                         "launch_bytes_frac": N ** 3 * (U1_STAGES * U1_RK_DESIGN_BYTES_PER_SITE_STAGE - 8 * 4) /
                                              (stage_s * U1_STAGES) / 1e9 / hbm_peak},
            "gpu_launches": launches, "clocks": clocks, "energies_end": energies_end,
            "gauss_tracking": "rms lattice Gauss charge of every step's starting state, summed in the first RK "
                              "stage (staged form) inside the timed steps"}


def rk_tiling(g, args, cl):
    """Apply --stages / --by / --dz to a Runge-Kutta lattice and return the tiling in effect
    (stages -1: the direct-load stage kernel)."""
    for opt, v in ((cl.CL_OPT_STAGES, args.stages), (cl.CL_OPT_TILE_BY, args.by), (cl.CL_OPT_TILE_DZ, args.dz)):
        if v is not None:
            g.cl_set_option(opt, v)
    return {"stages": g.cl_get_option(cl.CL_OPT_STAGES), "tile_by": g.cl_get_option(cl.CL_OPT_TILE_BY),
            "tile_dz": g.cl_get_option(cl.CL_OPT_TILE_DZ)}


def run_rk_workload(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src):
    """The headline two-field lattice advanced by the low-storage RK4-5 stages instead of the
    leapfrog (the non-symplectic evolver measured on the same 256^3 state)."""
    g = cl.Lattice(N, L, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_RK4_5, expansion=True, alpha=ALPHA, kappa=KAPPA, dt=DT,
                   stream=stream.cuda_stream)
    g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, G2])
    tiling = rk_tiling(g, args, cl)
    g.cl_init_vacuum(SEED, 1e30, AMP2, (1.0, 0.0), (0.0, 0.0))
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    el, launches, clocks = timed_region(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    e = g.cl_energies()
    g.close()
    stage_s = el / (args.steps * RK_STAGES)
    bytes_stage = N ** 3 * RK_BYTES_PER_SITE_STEP / RK_STAGES
    achieved = bytes_stage / stage_s / 1e9
    return {"metric": "Gsite-updates/s, 256^3 two fields, RK4-5", "value": world * N ** 3 * args.steps / el_max / 1e9,
            "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config({"workload": "two-field preheating m2phi2+g2phi2chi2, q=1e4, 256^3, RK4-5 (2N), "
                                          "FP32+Kahan, FP64 reductions, dt=0.005, self-consistent expansion",
                              "integrator": "rk4_5", "passes_per_step": RK_STAGES}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                         "kernel": ("k_rk_stage_tma<float,2,kahan,4,%d> (mean over the 5 stages)" % tiling["stages"]
                                    if tiling["stages"] > 0 else "k_rk_stage<float,2,kahan,4> (mean over the 5 stages)"),
                         "tiling": tiling,
                         "algorithmic_bytes_per_launch": bytes_stage},
            "gpu_launches": launches, "clocks": clocks,
            "energies_end": {"a": e["a"], "rho": e["rho"], "hubble_violation": e["hubble_violation"]}}


def run_reduced_workload(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src):
    """The headline's two-field model on a reduced (2+1)-dimensional lattice of 4096^2 sites
    (as many as 256^3), Yoshida-4, FP32 + Kahan: one launch of the reduced-lattice pass per
    pass.  The reduced lattices take no vacuum initial condition, so the state is the
    homogeneous phi = 1 plus seeded Gaussian noise of rms 1e-4 (phi, chi, their momenta)."""
    import numpy as np
    N2 = 4096
    L2 = 2048.0 * math.pi  # the headline's lattice spacing, pi / 32
    g = cl.Lattice(N2, L2, 2, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_YOSHIDA4, expansion=True, alpha=ALPHA, kappa=KAPPA,
                   dt=DT, stream=stream.cuda_stream, dims=2)
    g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, G2])
    if args.dz is not None:  # rows per chunk of the row-marching pass (tuning runs)
        g.cl_set_option(cl.CL_OPT_TILE_DZ, args.dz)
    if args.by is not None:  # rows ahead of its L2 prefetch (tuning runs)
        g.cl_set_option(cl.CL_OPT_TILE_BY, args.by)
    if args.variant is not None:  # 1: row marching (default), 0: one thread per site
        g.cl_set_option(cl.CL_OPT_PASS_VARIANT, args.variant)
    rng = np.random.default_rng(SEED)
    for f, (field, mom) in enumerate(((cl.CL_FIELD_PHI0, cl.CL_FIELD_PI0), (cl.CL_FIELD_PHI1, cl.CL_FIELD_PI1))):
        g.cl_set_state(field, ((1.0 if f == 0 else 0.0) + 1e-4 * rng.standard_normal((1, N2, N2))).astype(np.float32))
        g.cl_set_state(mom, (1e-4 * rng.standard_normal((1, N2, N2))).astype(np.float32))
    g.cl_set_scalars(1.0)
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    el, launches, clocks = timed_region(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    e = g.cl_energies()
    variant, rows = g.cl_get_option(cl.CL_OPT_PASS_VARIANT), g.cl_get_option(cl.CL_OPT_TILE_DZ)
    g.close()
    sites = N2 * N2
    pass_s = el / (args.steps * PASSES_PER_STEP)
    bytes_pass = sites * BYTES_PER_SITE_PASS
    achieved = bytes_pass / pass_s / 1e9
    return {"metric": "Gsite-updates/s, (2+1)-dimensional 4096^2 two fields, Yoshida-4",
            "value": world * sites * args.steps / el_max / 1e9,
            "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config({"workload": "two-field m2phi2+g2phi2chi2, q=1e4, reduced (2+1)-dimensional lattice "
                                          "4096^2, dx = pi/32, Yoshida-4, FP32+Kahan, FP64 reductions, dt=0.005, "
                                          "homogeneous phi=1 + noise 1e-4, self-consistent expansion",
                              "lattice": N2, "dims": 2, "integrator": "yoshida4", "passes_per_step": PASSES_PER_STEP,
                              "l2": "inputs (%.0f MB) larger than L2; no flush" % (sites * 24 / 1e6)}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                         "kernel": ("k_plane_pass<float,2,kahan,4> (row marching, %d rows a chunk; mean per pass)" % rows
                                    if variant == 1 else "k_reduced_pass<float,2,kahan> (mean per pass)"),
                         "algorithmic_bytes_per_launch": bytes_pass},
            "gpu_launches": launches, "clocks": clocks,
            "energies_end": {"a": e["a"], "rho": e["rho"], "hubble_violation": e["hubble_violation"]}}


def run_gw_workload(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src):
    """The headline two-field lattice with the gravitational-wave auxiliaries: every Yoshida-4
    pass is a GW pass (k_gw_pass) and the fused scalar pass."""
    g = make_lattice(cl, cl.CL_PREC_FP32_KAHAN, stream.cuda_stream)
    g.cl_enable_gw()
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    el, launches, clocks = timed_region(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    # the GW pass alone, timed over the same number of passes with the scalar pass removed by
    # difference: a second run of the scalar lattice without GW fields
    k, d, c = g.cl_gw_spectrum()
    g.close()
    g2 = make_lattice(cl, cl.CL_PREC_FP32_KAHAN, stream.cuda_stream)
    g2.cl_step(args.warmup)
    g2.cl_sync()
    el0, _, _ = timed_region(torch, g2, stream, args.steps)
    g2.close()
    gw_pass_s = max(el - el0, 1e-12) / (args.steps * PASSES_PER_STEP)
    bytes_gw = N ** 3 * GW_BYTES_PER_SITE_PASS
    achieved = bytes_gw / gw_pass_s / 1e9
    return {"metric": "Gsite-updates/s at 256^3 with gravitational waves", "value": world * N ** 3 * args.steps / el_max / 1e9,
            "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config({"workload": "two-field preheating as the headline, plus the five traceless GW "
                                          "auxiliaries (v, pi_v FP32) sourced by both fields, Yoshida-4",
                              "gw_fields": 10}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                         "kernel": "k_gw_pass<float,2,kahan,4> (time = with GW - without, per pass)",
                         "algorithmic_bytes_per_launch": bytes_gw},
            "scalar_only_ms_per_step": el0 / args.steps * 1e3,
            "gw_spectrum_bins": int(len(d)), "gw_rho_max_bin": float(d.max()),
            "gpu_launches": launches, "clocks": clocks}


def run_nmc_workload(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src):
    """One non-minimally coupled lambda phi^4 field at 256^3 with RK4-5: every stage is one
    launch of the TMA-staged stage kernel, which also sums the Ricci terms of its output state
    for the next stage (the direct-load kernel, --stages -1, needs a Ricci reduction launch
    before each stage)."""
    g = cl.Lattice(N, L, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_RK4_5, expansion=True, alpha=1.0, kappa=KAPPA, dt=DT,
                   stream=stream.cuda_stream)
    g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
    g.cl_init_vacuum(SEED, 16 * 2 * math.pi / L, 1e-4, (1.0,), (0.0,))
    g.cl_set_nonminimal(NMC_XI)
    tiling = rk_tiling(g, args, cl)
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    el, launches, clocks = timed_region(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    e = g.cl_energies()
    g.close()
    stage_s = el / (args.steps * RK_STAGES)
    bytes_stage = N ** 3 * NMC_BYTES_PER_SITE_STAGE
    achieved = bytes_stage / stage_s / 1e9
    return {"metric": "Gsite-updates/s at 256^3, non-minimally coupled field, RK4-5",
            "value": world * N ** 3 * args.steps / el_max / 1e9,
            "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config({"workload": "lambda phi^4 (program units), xi = %g, 256^3, RK4-5 (2N), FP32+Kahan, "
                                          "alpha = 1, vacuum amplitude 1e-4, k_cut = 16 k_IR" % NMC_XI,
                              "fields": 1, "integrator": "rk4_5", "passes_per_step": RK_STAGES}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                         "kernel": ("k_rk_stage_tma<float,1,kahan,4,%d> with the Ricci sums of its output (mean per stage)" % tiling["stages"]
                                    if tiling["stages"] > 0 else "k_nmc_ricci + k_rk_stage<float,1,kahan,4> (mean per stage)"),
                         "tiling": tiling,
                         "algorithmic_bytes_per_launch": bytes_stage},
            "ricci_end": e["ricci"], "gpu_launches": launches, "clocks": clocks}


def run_ensemble_workload(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src):
    import numpy as np
    c = dict(ENS)
    if args.members:  # smaller ensembles of the same mix (profiling runs)
        c["members"] = args.members
    rg = np.random.default_rng(c["seed"])
    sizes = [int(x) for x in rg.choice(c["sizes"], c["members"])]
    lam = 10.0 ** rg.uniform(math.log10(c["lam"][0]), math.log10(c["lam"][1]), c["members"])
    g = cl.Lattice(sizes[0], c["L"], 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_VV2, expansion=True, alpha=c["alpha"],
                   kappa=c["kappa"], dt=c["dt"], stream=stream.cuda_stream, member_N=sizes)
    g.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
    kcut = 16 * 2 * math.pi / c["L"]
    for m in range(c["members"]):  # lambda phi^4 in program units: lambda sets the vacuum amplitude
        g.cl_init_vacuum(c["seed"], kcut, float(lam[m]), (1.0,), (0.0,), member=m)
    sites = sum(n ** 3 for n in sizes)
    tuned = None
    if args.stages is None and args.by is None and args.dz is None and args.variant is None and not args.no_autotune:
        st_, by_, dz_, us_, var_ = g.cl_autotune()  # timed trial passes; the state is unchanged
        tuned = {"stages": st_, "tile_by": by_, "tile_dz": dz_, "variant": var_, "us_per_trial_pass": us_}
    for opt, v in ((cl.CL_OPT_PASS_VARIANT, args.variant), (cl.CL_OPT_STAGES, args.stages), (cl.CL_OPT_TILE_BY, args.by),
                   (cl.CL_OPT_TILE_DZ, args.dz)):
        if v is not None:
            g.cl_set_option(opt, v)
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    el, launches, clocks = timed_region(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    es = g.cl_energies(c["members"])
    tiles = {k: g.cl_get_option(o) for k, o in (("stages", cl.CL_OPT_STAGES), ("variant", cl.CL_OPT_PASS_VARIANT),
                                                ("member0_tile_by", cl.CL_OPT_TILE_BY),
                                                ("member0_tile_dz", cl.CL_OPT_TILE_DZ))}
    g.close()
    kname = ("k_ensemble_pass_tma<float,1,kahan,4,%d,%s>" % (tiles["stages"], "ringless" if tiles["variant"] else "ring")
             if tiles["stages"] > 0 else "k_ensemble_pass<float,1,kahan,4>")
    pass_s = el / args.steps
    bytes_pass = sites * ENS_BYTES_PER_SITE
    achieved = bytes_pass / pass_s / 1e9
    return {"metric": "Gsite-updates/s, ensemble of %d lattices" % c["members"], "value": world * sites * args.steps / el_max / 1e9,
            "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d lambda phi^4 lattices, N from {32,48,64} (seeded), vacuum amplitude " % c["members"] +
                                   "log-uniform in [1e-6,1e-3], L=8 pi, VV-2, FP32+Kahan, dt=0.01",
                       "members": c["members"], "sites": sites,
                       "l2": "inputs (%.0f MB) larger than L2; no flush" % (sites * 6 * 4 / 1e6)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                         "kernel": kname, "tiles": tiles, "algorithmic_bytes_per_launch": bytes_pass},
            "autotune": tuned,
            "gpu_launches": launches, "clocks": clocks,
            "energies_end": {"members": len(es), "max_hubble_violation": max(x["hubble_violation"] for x in es),
                             "steps": es[0]["step"]}}


SG = dict(N=128, cin=3, cout=2, hidden=48, layers=6, K=16, seed=1234)


def surrogate_flops(N, cin, cout, hidden, layers):
    """Multiply-adds x 2 of one forward: 27 taps per input-output channel pair and site."""
    pairs = cin * hidden + (layers - 2) * hidden * hidden + hidden * cout
    return 2 * 27 * pairs * N ** 3


def run_surrogate_workload(args, world, rank, local, cl, torch, stream, peak_tf, peak_src):
    import numpy as np
    c = SG
    N = c["N"]
    rg = np.random.default_rng(c["seed"])

    def build(layers):
        s = cl.Surrogate(N, c["cin"], c["cout"], c["hidden"], layers, cl.CL_ACT_RELU, cl.CL_SG_BF16,
                         stream=stream.cuda_stream)
        for l, (ci, co) in enumerate(s.shapes):
            s.set_weights(l, rg.standard_normal((27, co, ci)) * math.sqrt(2.0 / (27 * ci)), 0.01 * rg.standard_normal(co))
        return s

    x = torch.randn(N ** 3 * c["cin"], device="cuda", dtype=torch.float32)
    y = torch.empty(N ** 3 * c["cout"], device="cuda", dtype=torch.float32)
    g = torch.randn(N ** 3 * c["cout"], device="cuda", dtype=torch.float32)

    def time_it(fn, n):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3 / n

    s6 = build(c["layers"])
    s2 = build(2)
    clk = Clocks(local)
    with clk:
        t6 = time_it(lambda: s6.forward(x, y), args.steps)
        t2 = time_it(lambda: s2.forward(x, y), args.steps)
        tfb = time_it(lambda: (s6.forward(x, y), s6.backward(g)), max(2, args.steps // 10))
    launches = s6.last_launch_count()
    s6.close()
    s2.close()
    # the leapfrog steps one forward replaces: K VV-2 steps, one field, FP32 + Kahan, 128^3, each
    # time K steps queued by one cl_step call (graph replays), timed on the device
    lat = cl.Lattice(N, 8.0 * math.pi * N / 256, 1, cl.CL_PREC_FP32_KAHAN, cl.CL_INT_VV2, alpha=1.0, kappa=0.1,
                     dt=0.01, stream=stream.cuda_stream)
    lat.cl_set_potential(cl.CL_POT_LPHI4, [1.0])
    lat.cl_init_vacuum(c["seed"], 1e30, 1e-4, (1.0,), (0.0,))
    lat.cl_step(20)
    lat.cl_sync()
    tl = time_it(lambda: lat.cl_step(c["K"]), 20)
    lf_tiles = {k: lat.cl_get_option(o) for k, o in (("tile_by", cl.CL_OPT_TILE_BY), ("tile_dz", cl.CL_OPT_TILE_DZ),
                                                     ("stages", cl.CL_OPT_STAGES), ("variant", cl.CL_OPT_PASS_VARIANT))}
    lat.close()
    # break-even: the forward time of each hidden width against the leapfrog step, i.e. the jump
    # length K at which one forward costs as much as the K steps it replaces
    breakeven = {}
    for hid in (16, 32, 48):
        sv = cl.Surrogate(N, c["cin"], c["cout"], hid, c["layers"], cl.CL_ACT_RELU, cl.CL_SG_BF16,
                          stream=stream.cuda_stream)
        for l, (ci, co) in enumerate(sv.shapes):
            sv.set_weights(l, rg.standard_normal((27, co, ci)) * math.sqrt(2.0 / (27 * ci)), 0.01 * rg.standard_normal(co))
        tf = time_it(lambda: sv.forward(x, y), max(5, args.steps))
        sv.close()
        breakeven[str(hid)] = {"forward_ms": tf * 1e3, "flops": surrogate_flops(N, c["cin"], c["cout"], hid, c["layers"]),
                               "breakeven_K": tf / (tl / c["K"])}
    flops = surrogate_flops(N, c["cin"], c["cout"], c["hidden"], c["layers"])
    tc_flops = 2 * 27 * c["hidden"] ** 2 * N ** 3
    tc_s = (t6 - t2) / (c["layers"] - 2)
    achieved = tc_flops / tc_s / 1e12
    # a bounded training run and the judged jumps (the learned path end to end)
    from paper_2607_24978_gb300 import surrogate_train as T
    trained = {}
    if not args.no_train:
        for hid, K in ((c["hidden"], c["K"]), (32, 32)):  # the configured network, a cheaper break-even variant
            with torch.cuda.stream(stream):
                st, mu, sg, info = T.train(torch, N=32, hidden=hid, K=K, iters=2000, lr=1e-4)
                ev = {n: T.evaluate(torch, st, mu, sg, N=n, K=K, jumps=8, hubble_limit=1e-3, hidden=hid)
                      for n in (64, 128)}
                ev_free = T.evaluate(torch, st, mu, sg, N=128, K=K, jumps=8, hubble_limit=float("inf"), hidden=hid)
                st.close()
            e128 = ev[128]
            ok = e128["accepted"] == e128["jumps"] and max(e128["spectrum_err_phi"], e128["spectrum_err_pi"]) <= 0.01
            trained["hidden%d_K%d" % (hid, K)] = {
                "training": info, "judged_jumps": {str(k): v for k, v in ev.items()},
                "unjudged_jumps_128": ev_free,
                "surrogate_speedup_at_1pct_err": e128["speedup"] if ok else None}
        trained["note"] = ("speed-up at 1 % spectrum error reported only when every jump is accepted and both "
                           "binned spectra are within 1 % of the plain leapfrog")
    return {"metric": "surrogate forward TFLOP/s at 128^3 (6 layers, 48 channels, BF16)", "value": flops / t6 / 1e12,
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t6 * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "periodic 3x3x3 conv surrogate 3->48->48x4->2, ReLU, residual jump, 128^3, "
                                   "BF16 tensor cores (FP32 accumulation); random weights",
                       "flops_per_forward": flops, "l2": "activations (201 MB per hidden layer) larger than L2"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": achieved / peak_tf, "traffic": None, "peak_source": peak_src,
                         "kernel": "k_conv_tc<48> (one hidden layer; time = (6-layer - 2-layer forward) / 4)",
                         "algorithmic_flops_per_launch": tc_flops},
            "forward_backward": {"ms": tfb * 1e3, "tflops": 3 * flops / tfb / 1e12},
            "leapfrog": {"steps": c["K"], "ms": tl * 1e3, "ms_per_step": tl / c["K"] * 1e3,
                         "GBps_per_pass": N ** 3 * ENS_BYTES_PER_SITE / (tl / c["K"]) / 1e9, "tiles": lf_tiles,
                         "forward_over_leapfrog": t6 / tl},
            "breakeven_by_hidden_width": breakeven,
            "trained": trained,
            "gpu_launches": launches, "clocks": clk.summary()}


# ------------------------------------------------------------------ GPU arm
def make_lattice(cl, precision, stream, args=None, n=None):
    n = N if n is None else n  # other sizes keep the lattice spacing of the 256^3 box
    g = cl.Lattice(n, L * n / 256, 2, precision, cl.CL_INT_YOSHIDA4, expansion=True, alpha=ALPHA, kappa=KAPPA,
                   dt=DT, stream=stream)
    g.cl_set_potential(cl.CL_POT_M2_G2, [1.0, G2])
    g.cl_init_vacuum(SEED, 1e30, AMP2, (1.0, 0.0), (0.0, 0.0))
    if args is not None:  # tile overrides (profiling and tuning runs)
        if args.stages is not None:
            g.cl_set_option(cl.CL_OPT_STAGES, args.stages)
        if args.by is not None:
            g.cl_set_option(cl.CL_OPT_TILE_BY, args.by)
        if args.dz is not None:
            g.cl_set_option(cl.CL_OPT_TILE_DZ, args.dz)
        if args.variant is not None:
            g.cl_set_option(cl.CL_OPT_PASS_VARIANT, args.variant)
    return g


def timed_steps(torch, g, stream, steps):
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    g.cl_sync()
    start.record(stream)
    launches = 0
    for _ in range(steps):
        g.cl_step(1)
        launches += g.cl_last_launch_count()
    stop.record(stream)
    stop.synchronize()
    g.cl_sync()
    return start.elapsed_time(stop) / 1e3, launches


def e2e_leg(args, world, cl, torch, g):
    """The headline metric through the C ABI with host buffers, and the transfer rates it sees
    beside plain pinned cudaMemcpyAsync copies (torch) of the same arrays."""
    nsite = N ** 3
    steps = max(3, min(args.steps, 10))
    tdt = torch.float64 if args.precision == "fp64" else torch.float32
    es = 8 if args.precision == "fp64" else 4
    host_in = [torch.empty(nsite, dtype=tdt, pin_memory=True) for _ in range(4)]
    host_out = [torch.empty(nsite, dtype=tdt, pin_memory=True) for _ in range(4)]
    fields = [cl.CL_FIELD_PHI0, cl.CL_FIELD_PHI1, cl.CL_FIELD_PI0, cl.CL_FIELD_PI1]
    for h, f in zip(host_in, fields):
        g.cl_get_state(f, h.numpy())
    a_in = [h.numpy() for h in host_in]
    a_out = [h.numpy() for h in host_out]
    g.cl_sync()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        for a, f in zip(a_in, fields):
            g.cl_set_state(f, a)
        g.cl_step(1)
        for a, f in zip(a_out, fields):
            g.cl_get_state(f, a)
        g.cl_energies()
    el = max_over_ranks(time.perf_counter() - t0, world)
    # the transfers alone through the same calls, and plain pinned copies of the same bytes
    t0 = time.perf_counter()
    for a, f in zip(a_in, fields):
        g.cl_set_state(f, a)
    g.cl_sync()
    t_up = time.perf_counter() - t0
    t0 = time.perf_counter()
    for a, f in zip(a_out, fields):
        g.cl_get_state(f, a)
    t_down = time.perf_counter() - t0
    dev = [torch.empty(nsite, dtype=tdt, device="cuda") for _ in range(4)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for d, h in zip(dev, host_in):
        d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    p_up = time.perf_counter() - t0
    t0 = time.perf_counter()
    for d, h in zip(dev, host_out):
        h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    p_down = time.perf_counter() - t0
    del dev
    nbytes = 4 * nsite * es
    return {"value": world * nsite * steps / el / 1e9, "unit": "Gsite-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 14 * 8, "steps": steps,
            "ms_per_step": el / steps * 1e3,
            "path": "cl_set_state x4 (pinned host) + cl_step(1) + cl_get_state x4 (pinned host) + cl_energies",
            "h2d_GBps": nbytes / t_up / 1e9, "d2h_GBps": nbytes / t_down / 1e9,
            "plain_pinned_copy_h2d_GBps": nbytes / p_up / 1e9, "plain_pinned_copy_d2h_GBps": nbytes / p_down / 1e9}


def size_point(args, cl, torch, stream, n, hbm_peak, peak_src):
    """The headline workload at n^3 (same model and spacing): throughput and the fused pass's
    roofline fraction."""
    g = make_lattice(cl, cl.CL_PREC_FP32_KAHAN, stream.cuda_stream, n=n)
    g.cl_step(3)
    g.cl_sync()
    steps = max(args.steps, 20)
    el, launches = timed_steps(torch, g, stream, steps)
    e = g.cl_energies()
    tiles = {k: g.cl_get_option(o) for k, o in (("tile_by", cl.CL_OPT_TILE_BY), ("tile_dz", cl.CL_OPT_TILE_DZ),
                                                ("stages", cl.CL_OPT_STAGES), ("variant", cl.CL_OPT_PASS_VARIANT))}
    g.close()
    bytes_launch = n ** 3 * BYTES_PER_SITE_PASS
    achieved = bytes_launch / (el / (steps * PASSES_PER_STEP)) / 1e9
    return {"lattice": n, "value": n ** 3 * steps / el / 1e9, "unit": "Gsite-updates/s", "steps": steps,
            "ms_per_step": el / steps * 1e3, "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_source": peak_src, "tiles": tiles,
                         "algorithmic_bytes_per_launch": bytes_launch},
            "hubble_violation_end": e["hubble_violation"],
            "l2": "inputs (%.1f GB) larger than L2; no flush" % (n ** 3 * 6 * 4 / 1e9)}


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2607_24978_gb300 import build_ext, cl
    build_ext.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    peaks = load_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "of measured" if peaks else "of fallback"
    if args.workload == "surrogate":
        tf = peaks["bf16_tflops"] if peaks else 1900.0
        line = run_surrogate_workload(args, world, rank, local, cl, torch, stream, tf,
                                      "of measured" if peaks else "of fallback")
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload != "preheat":
        fn = {"u1": run_u1_workload, "rk": run_rk_workload, "gw": run_gw_workload,
              "u1lf": lambda *a: run_u1_workload(*a, leapfrog=True),
              "nmc": run_nmc_workload, "reduced": run_reduced_workload}.get(args.workload, run_ensemble_workload)
        line = fn(args, world, rank, local, cl, torch, stream, hbm_peak, peak_src)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    prec = {"fp32k": cl.CL_PREC_FP32_KAHAN, "fp64": cl.CL_PREC_FP64, "fp32": cl.CL_PREC_FP32}[args.precision]
    g = make_lattice(cl, prec, stream.cuda_stream, args)
    g.cl_step(args.warmup)
    g.cl_sync()
    barrier(world)
    clk = Clocks(local)
    with clk:
        el, launches = timed_steps(torch, g, stream, args.steps)
    barrier(world)
    el_max = max_over_ranks(el, world)
    value = world * N ** 3 * args.steps / el_max / 1e9
    e = g.cl_energies()

    # roofline of the dominant kernel: the fused scalar pass, PASSES_PER_STEP launches per step
    pass_s = el / (args.steps * PASSES_PER_STEP)
    bytes_site = {"fp32k": BYTES_PER_SITE_PASS, "fp64": BYTES_PER_SITE_PASS_FP64, "fp32": 2 * 2 * 2 * 4}[args.precision]
    bytes_launch = N ** 3 * bytes_site
    achieved = bytes_launch / pass_s / 1e9
    traffic = profiled_traffic() if args.precision == "fp32k" and N == 256 else None
    tiles = {k: g.cl_get_option(o) for k, o in (("tile_by", cl.CL_OPT_TILE_BY), ("tile_dz", cl.CL_OPT_TILE_DZ),
                                                ("stages", cl.CL_OPT_STAGES), ("variant", cl.CL_OPT_PASS_VARIANT))}
    kname = ("k_scalar_pass_tma_nr" if tiles["variant"] == 1 else "k_scalar_pass_tma") if tiles["stages"] > 0 \
        else "k_scalar_pass"
    tname = {"fp32k": "float,2,kahan,4", "fp64": "double,2,plain,2", "fp32": "float,2,plain,4"}[args.precision]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic, "kernel": "%s<%s,%d>" % (kname, tname, tiles["stages"]), "tiles": tiles,
                "algorithmic_bytes_per_launch": bytes_launch, "peak_source": peak_src}

    if args.profile:
        print(json.dumps({"metric": METRIC, "value": value, "unit": "Gsite-updates/s", "profile": True,
                          "steps": args.steps, "roofline_frac": roofline["frac"],
                          "gpu_launches": launches}), flush=True)
        g.close()
        return

    # end to end through the C ABI with host buffers: every step uploads phi and pi of both
    # fields from pinned host memory, advances one step and reads phi, pi and the energies back
    e2e = e2e_leg(args, world, cl, torch, g)
    g.close()

    # the config's 512^3 roofline point (same model and spacing, 8x the sites)
    big = None
    if N != 512 and not args.no_512:
        big = size_point(args, cl, torch, stream, 512, hbm_peak, peak_src)

    # the same workload in FP64 without compensation ("FP64 plain")
    g64 = make_lattice(cl, cl.CL_PREC_FP64, stream.cuda_stream)
    g64.cl_step(2)
    n64 = max(2, min(args.steps, 10))
    el64, _ = timed_steps(torch, g64, stream, n64)
    g64.close()
    fp64 = {"value": N ** 3 * n64 / el64 / 1e9, "unit": "Gsite-updates/s", "steps": n64,
            "fp32_kahan_speedup": (N ** 3 * args.steps / el) / (N ** 3 * n64 / el64),
            "achieved_GBps": N ** 3 * BYTES_PER_SITE_PASS_FP64 / (el64 / (n64 * PASSES_PER_STEP)) / 1e9}
    # the FP64 pass is bound by the FP64 pipe (2 FP64 operations per SM per cycle on GB300), not by HBM
    rec = fp64_ops_record()
    if rec is not None:
        peak = rec["fp64_peak_ops_per_cycle_per_sm"] * rec["sm_count"] * rec["sm_max_mhz"] * 1e6
        ach = rec["fp64_ops_per_site_pass"] * N ** 3 * PASSES_PER_STEP * n64 / el64
        fp64["roofline"] = {"bound": "alu", "achieved": ach / 1e9, "peak": peak / 1e9, "unit": "G FP64 op/s",
                            "frac": ach / peak, "kernel": rec["kernel"],
                            "ops_per_site_pass": rec["fp64_ops_per_site_pass"],
                            "peak_source": "2 FP64 ops per SM per cycle (ncu peak_sustained) x 152 SMs x 2070 MHz"}

    line = {"metric": METRIC, "value": value, "unit": "Gsite-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": config({"parallelism": "replicas" if world > 1 else "single", "precision": args.precision}),
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
            "fp64_plain": fp64, "energies_end": {"a": e["a"], "rho": e["rho"], "hubble_violation": e["hubble_violation"]}}
    if big is not None:
        line["lattice_512"] = big
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 1000; 200 oracle steps of the reference arm)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="time the device steps only (no e2e, FP64 or CPU legs): the command profiled with ncu")
    ap.add_argument("--stages", type=int, default=None, help="override CL_OPT_STAGES")
    ap.add_argument("--by", type=int, default=None, help="override CL_OPT_TILE_BY")
    ap.add_argument("--dz", type=int, default=None, help="override CL_OPT_TILE_DZ")
    ap.add_argument("--variant", type=int, default=None,
                    help="override CL_OPT_PASS_VARIANT (scalar pass: 0 ring, 1 ringless; U(1): 0 gather, 1 fused, 2 staged)")
    ap.add_argument("--workload", default="preheat", choices=["preheat", "u1", "u1lf", "ensemble", "surrogate", "rk", "gw", "nmc",
                                                              "reduced"],
                    help="preheat: the headline 256^3 two-field run; u1, ensemble: the other workloads")
    ap.add_argument("--members", type=int, default=None, help="ensemble size (default 1024)")
    ap.add_argument("--no-train", action="store_true", help="surrogate workload: throughput only")
    ap.add_argument("--no-autotune", action="store_true", help="ensemble workload: default tiling, no trial passes")
    ap.add_argument("--lattice", type=int, default=256,
                    help="preheat workload: sites per side (same model and lattice spacing as 256^3)")
    ap.add_argument("--no-512", action="store_true", help="preheat workload: skip the 512^3 roofline point")
    ap.add_argument("--precision", default="fp32k", choices=["fp32k", "fp64", "fp32"],
                    help="preheat workload: FP32 + Kahan (default), FP64, or plain FP32")
    args = ap.parse_args()
    global N, METRIC
    if args.lattice != N:
        N = args.lattice
        METRIC = "Gsite-updates/s at %d^3" % N
    if args.steps is None:
        args.steps = 200 if args.impl == "reference" else 1000
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
