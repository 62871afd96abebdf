"""Benchmark: time to an FP64 true residual ||b - D x||/||b|| <= 1e-10 per
right-hand side for the adaptive-multigrid Wilson-clover solver.

Headline workload (the largest single-GPU configuration; synthetic stand-in
for the paper's gauge ensembles): a 48^3 x 96 lattice, links exp(0.5 i H)
(seed 4), kappa = 0.129, c_sw = 1.0, antiperiodic in t; the 12 spin-colour
point sources at the origin; two-level multigrid with 4^4 blocks and 24 test
vectors (48 chiral), FP32 smoother, bfloat16 coarse operator whose batched
coarse solves run their stencil on the tensor cores, test vectors stored in
half precision with a per-site scale for restriction and prolongation, FP64
outer flexible GMRES(8).  The gauge field and the initial test vectors
are drawn on the device by the library's counter-based generator.
One step = one call of amg_solve on all 12 sources (x = 0 each time).  The
setup (test vectors, Galerkin operator) runs once before the timed region and
is reported separately.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload instead; ``--workload`` selects the
secondary workloads (solve16, dirac, mixed3, ragged, coarse_tc, learned).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lqcd_inputs as li  # noqa: E402

METRIC = "time to FP64 |r|/|b|<=1e-10 per RHS; Dirac/coarse matvec % HBM/TC roofline"
TOL = 1e-10
# the headline workload: 12 spin-colour point sources on 48^3 x 96
PROP = dict(dims=(48, 48, 48, 96), eps=0.5, seed=4, kappa=0.129, csw=1.0, block=(4, 4, 4, 4), nvec=24, outer_m=8,
            nsrc=12)
PROP_CONFIG = {
    "workload": "48^3x96 Wilson-clover (exp(0.5iH) links, seed 4, kappa 0.129, csw 1.0, antiperiodic t), "
                "12 spin-colour point sources at the origin per step; 2-level AMG, 4^4 blocks, 24 test vectors "
                "(n_init 3, n_adapt 2), SAP(4) x MR(6) smoother, BiCGStab(2) coarse solve to 1e-2, "
                "FP64 outer flexible GMRES(8) to a true residual of 1e-10",
    "lattice": [48, 48, 48, 96], "rhs_per_step": 12,
    "precision": "FP32 smoother, bfloat16 coarse operator with the batched coarse solves' stencil on the tensor "
                 "cores (tcgen05, FP32 accumulation), FP16 test vectors (per-site scale) in restriction and "
                 "prolongation, FP64 outer solver (Gram-Schmidt and true residual in FP64; Arnoldi products "
                 "and the solution update in FP64-accurate double-float pair arithmetic)",
    "l2": "working set > L2 (no flush)",
}
# a second workload kept for comparison with earlier measurements: one Gaussian source on 16^3 x 32
SOLVE16 = dict(dims=(16, 16, 16, 32), eps=0.6, seed=2, kappa=0.130, csw=1.0, block=(4, 4, 4, 4), nvec=24)
# the sub-lattice on which the CPU oracle samples the headline workload (same eps, seed, kappa, c_sw, blocking)
ORACLE_SAMPLE_DIMS = (8, 8, 8, 8)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _fp32_fma_peak(torch):
    """FP32 FMA peak in TFLOP/s from the device's SM count (128 FP32 lanes per
    SM, 2 flop per FMA) and the maximum SM clock (measured file, else 2070 MHz)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


class ClockSampler:
    """Continuous nvidia-smi sampling (every 100 ms) around the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.samples = []
        self._p = None
        self._t = None

    def _reader(self):
        for line in self._p.stdout:
            parts = [x.strip() for x in line.strip().split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __enter__(self):
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self._p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                        "-lms", "100", "-i", dev], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                       text=True)
            self._t = threading.Thread(target=self._reader, daemon=True)
            self._t.start()
            t0 = time.time()
            while not self.samples and time.time() - t0 < 5:
                time.sleep(0.05)
        except Exception:
            self._p = None
        return self

    def __exit__(self, *a):
        if self._p is not None:
            time.sleep(0.15)
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
            self._t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(s[1]) for s in self.samples) if v is not None]
        mx = [v for v in (num(s[2]) for s in self.samples) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[4 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(x, world):
    """The largest x over the ranks of the default process group (x for one
    rank): the job's time is the slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


SAP_DRAM_BYTES_PER_SITE_RHS = 1378.0
SAP_KERNEL_NAMES = {0: "sap_half_kernel<P32,256> (fused SAP half sweep)",
                    1: "sap_half_staged_kernel<P32> (fused SAP half sweep, operator staged in shared memory)",
                    2: "sap_half_kernel<P32,256,2> (fused SAP half sweep, two right-hand sides per CTA)",
                    3: "sap_half_staged_kernel<P32,P16> (fused SAP half sweep, FP16 operator staged in shared memory)"}


def make_params(capi, prec_smoother, coarse="f32", outer="fgmres", sap_variant=-1, setup=None, vec="f32", w=None):
    p = capi.amg_params_default()
    if vec == "f16":
        p.prec_vectors = capi.AMG_F16
    p.outer_solver = {"fgmres": 0, "fbicgstab": 1, "mbicgs": 2}[outer]
    p.sap_variant = sap_variant
    for k, v in (setup or {}).items():
        if v is not None:
            setattr(p, k, v)
    p.nlevels = 2
    for mu in range(4):
        p.block[0][mu] = w["block"][mu]
    p.nvec[0] = w["nvec"]
    p.prec_smoother = prec_smoother
    if prec_smoother == capi.AMG_F64:
        p.prec_coarsest = capi.AMG_F64
    else:
        p.prec_coarsest = capi.AMG_BF16 if coarse == "bf16" else capi.AMG_F32
    return p


def timed_cores(fn):
    """Run fn(); returns (its result, wall seconds, cores used), the cores being
    the process CPU time over the wall time, at least 1."""
    w0, c0 = time.perf_counter(), time.process_time()
    out = fn()
    wall, cpu = time.perf_counter() - w0, time.process_time() - c0
    return out, wall, max(1, int(round(cpu / wall))) if wall > 0 else 1


# ---- the FP64 CPU oracle on a bounded sample of the headline workload ------------------
# A sample is one outer iteration's dominant work on the 8^4 sub-lattice of the headline
# workload (same eps, seed, kappa, c_sw, 4^4 blocks, 24 test vectors): one application of
# the multigrid preconditioner (restrict, coarse BiCGStab(2), prolong, SAP) and one fine D,
# on point source k mod 12.  The oracle's hierarchy is built from orthonormalised seeded
# vectors (its adaptive setup takes minutes at this size; the cost of a cycle does not depend
# on the vectors' quality).  Samples run in one single-threaded worker process per host core
# (independent right-hand sides), started with spawn.

_ORACLE = {}


def _oracle_init():
    from oracle import dirac as odirac, amg as oamg
    w, dims = PROP, ORACLE_SAMPLE_DIMS
    U = li.gauge_field(dims, w["eps"], w["seed"])
    op = odirac.WilsonClover(U, w["kappa"], w["csw"], True)
    shape4 = li.lattice_shape(dims)
    v0 = li.test_vectors(dims, w["seed"], w["nvec"]).reshape((w["nvec"],) + shape4 + (12,))
    hier = oamg.Hierarchy(op, oamg.AMGParams(blocks=[w["block"]], nvecs=[w["nvec"]]))
    hier.set_vectors([v0])
    _ORACLE.update(op=op, hier=hier, shape4=shape4)


def _oracle_sample(k):
    op, hier, shape4 = _ORACLE["op"], _ORACLE["hier"], _ORACLE["shape4"]
    b = li.point_source(ORACLE_SAMPLE_DIMS, (k % 12) // 3, k % 3).reshape(shape4 + (12,))
    t0 = time.perf_counter()
    z = hier.vcycle(0, b)
    op.apply(z)
    return time.perf_counter() - t0


class OraclePool:
    """spawn-started worker processes, one per host core, each single-threaded
    (BLAS threads pinned to 1) with its own copy of the sample hierarchy."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.procs = procs or (os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init)

    def run(self, nsamples, first=0):
        """Wall seconds for nsamples samples spread over the workers."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_sample, range(first, first + nsamples), chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_extrapolation(wall, nsamples, cycles):
    """ms per right-hand side of the full workload from the sample throughput:
    (wall / samples) x preconditioner applications per RHS x volume ratio."""
    vol = float(np.prod(PROP["dims"])) / float(np.prod(ORACLE_SAMPLE_DIMS))
    return wall / nsamples * cycles * vol * 1e3


def _sample_text(procs, nsamples, cycles, cycles_from):
    return (f"{nsamples} samples on the 8^4 sub-lattice of the workload (same eps, seed, kappa, c_sw, blocking; "
            f"one sample = one FP64 oracle multigrid cycle + one D on a point source) in {procs} single-threaded "
            f"spawn workers (one per host core, independent sources); extrapolated: wall/sample x "
            f"{cycles:g} preconditioner applications per RHS ({cycles_from}) x "
            f"{np.prod(PROP['dims']) // np.prod(ORACLE_SAMPLE_DIMS)} (volume ratio)")


# preconditioner applications per right-hand side the method needs on the headline workload
# (four outer flexible GMRES steps, measured by the GPU arm); the oracle arm runs in its own
# process and cannot see the GPU arm's live count
HEADLINE_CYCLES = 4


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    pool = OraclePool()
    # one step = one sample per host core (all cores busy); warm-up steps first, at least one
    # (every worker builds its sample hierarchy then)
    per_step = pool.procs
    warm = max(args.warmup, 1)
    pool.run(warm * per_step)
    nsamp = args.steps * per_step
    wall = pool.run(nsamp, first=warm * per_step)
    pool.close()
    per_rhs_ms = oracle_extrapolation(wall, nsamp, HEADLINE_CYCLES)
    cpu = {"value": per_rhs_ms, "unit": "ms/RHS", "cores": pool.procs, "kind": "oracle",
           "sample": _sample_text(pool.procs, nsamp, HEADLINE_CYCLES, "the count the GPU solve measures")}
    line = {
        "impl": "reference", "metric": METRIC, "value": per_rhs_ms, "unit": "ms/RHS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": warm, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": PROP_CONFIG, "cpu_baseline": cpu,
        "e2e": {"value": per_rhs_ms, "unit": "ms/RHS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "details": {"steps_are": f"{per_step} oracle samples each, one per host core in parallel "
                                 "(ms_per_step = wall time of the timed samples / steps)",
                    "extrapolated": True},
    }
    print(json.dumps(line), flush=True)


def _point_sources(torch, V, nsrc):
    """nsrc canonical FP64 fields on the device: source k = delta at the origin, spin k // 3, colour k % 3."""
    b = torch.zeros(nsrc * V * 24, dtype=torch.float64, device="cuda")
    for k in range(nsrc):
        b[k * V * 24 + 2 * k] = 1.0        # site 0, (spin, colour) index k, real part
    return b


def run_headline(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_info()
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.dims:
        pool = OraclePool()      # spawn before the first GPU call; workers build their samples meanwhile
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi

    w = dict(PROP)
    config = PROP_CONFIG
    if args.dims:   # a smaller lattice of the same workload (profiling); the config says so
        w["dims"] = tuple(int(v) for v in args.dims.split(","))
        config = dict(PROP_CONFIG, lattice=list(w["dims"]),
                      workload=PROP_CONFIG["workload"].replace("48^3x96", "x".join(map(str, w["dims"]))))
    if args.resid_pair:
        config = dict(config, precision=config["precision"].replace(
            "Gram-Schmidt and true residual in FP64; Arnoldi products and the solution update",
            "Gram-Schmidt in FP64; Arnoldi products, the true residual and the solution update"))
    dims = w["dims"]
    V = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    lat = capi.amg_lattice_create(dims, True)
    g = capi.amg_gauge_random(lat, w["eps"], w["seed"])
    d = capi.amg_dirac_create(g, w["kappa"], w["csw"])
    init = torch.empty(w["nvec"] * V * 24, dtype=torch.float64, device="cuda")
    capi.amg_random_normal(w["seed"] + 2000, li.STREAM_TESTVEC, 0, w["nvec"] * V * 12, init)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    p = make_params(capi, capi.AMG_F32, vec="f16", w=w, sap_variant=args.sap_variant)
    p.outer_m = w["outer_m"]
    p.sap_eo = 1 if args.sap_eo else 0
    if args.mr is not None:
        p.mr_iters = args.mr
    if args.prop_coarse == "bf16":
        p.prec_coarsest = capi.AMG_BF16
        p.coarse_tc = 0 if args.no_coarse_tc else 1
    p.resid_pair = 1 if args.resid_pair else 0
    t0 = time.perf_counter()
    h = capi.amg_setup(d, p, [init])
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    del init
    torch.cuda.empty_cache()
    ns = w["nsrc"]
    b = _point_sources(torch, V, ns)
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        x.zero_()
        capi.amg_solve(h, b, x, ns, TOL, 200, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    infos = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler() as clk:
        torch.cuda.nvtx.range_push("timed")
        l0 = capi.amg_launch_count()
        ev0.record(stream)
        for _ in range(args.steps):
            x.zero_()
            st, info = capi.amg_solve(h, b, x, ns, TOL, 200, stream=stream)
            infos.append(info.as_dict())
        ev1.record(stream)
        gpu_launches = capi.amg_launch_count() - l0
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms / args.steps
    per_rhs = ms / (args.steps * ns * world)
    ok = all(i["converged"] == 1 and i["true_rel_residual"] <= TOL for i in infos)

    # end to end through the public API: amg_solve on the step's sources and solutions in
    # pinned host memory (the library copies each batch in and out on its copy stream,
    # overlapped with the neighbouring batches' solves), copies inside the timed region
    ne2e = max(1, min(args.steps, 2))
    hb = b.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    capi.amg_solve(h, hb, hx, ns, TOL, 200, stream=stream)   # untimed: allocates the copy staging once
    torch.cuda.synchronize()
    e2e_infos = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(ne2e):
        st_, inf_ = capi.amg_solve(h, hb, hx, ns, TOL, 200, stream=stream)
        e2e_infos.append(inf_.as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / (ne2e * ns)
    # the host solutions against the device ones of the timed steps (same sources)
    xd = x.cpu()
    e2e_diff = float((hx - xd).abs().max() / xd.abs().max())
    del xd
    del hb, hx

    # dominant kernel: the fused SAP half sweep (one launch = one colour of domains, every
    # right-hand side of a batch).  Algorithmic work per active site: the residual b - D x
    # (1872 + 24 flop) and mr_iters minimal-residual steps on D_SAP (1494 flop for the
    # in-domain hops and clover of a 4^4 domain + 336 for two dot products and two updates);
    # half the sites are active per colour.  Average launch time from the library's CUDA-event
    # smoother timer over the timed region.
    peak, sms, mhz = _fp32_fma_peak(torch)
    cycles = float(np.mean([i["cycles"] for i in infos]))
    smooth_ms = float(np.mean([i["ms_smoother"] for i in infos]))
    if p.sap_eo:
        # even-odd domain solves: residual (1872 + 24), the Schur right-hand side and the odd
        # reconstruction (each in-domain hops + one clover (inverse) on one site of a pair:
        # 1494 per pair = 747 per site, twice), and per minimal-residual step the four
        # parity blocks (hops and clover (inverse) on both sites of a pair, 2988) plus the
        # dots and updates on the even site (336): 1578 per site
        flop_site = 1872 + 24 + 2 * 747 + p.mr_iters * 1578
    else:
        flop_site = 1872 + 24 + p.mr_iters * (1494 + 336)
    flop_step = flop_site * (V / 2) * 2 * p.sap_iters * cycles * ns
    sap_tflops = flop_step / (smooth_ms * 1e-3) / 1e12
    # DRAM traffic of one launch (one colour, the batch's right-hand sides), scaled from an ncu
    # capture of sap_half_kernel<P32,256,1> on 24^3x48 with 12 right-hand sides per launch
    # (dram__bytes_read.sum + dram__bytes_write.sum = 2.372 + 0.371 GB over 165,888 active sites x
    # 12 right-hand sides = 1378 B per active site and right-hand side); variant 0 only
    width = max(int(i.get("batch_width", 0)) for i in infos) or 1
    sap_traffic = (SAP_DRAM_BYTES_PER_SITE_RHS * (V / 2) * width
                   if (args.sap_variant == 0 and not p.sap_eo) else None)
    hbm, kind = _peaks()
    # the other kernels the metric names, timed alone on this workload's fields
    kern = {}
    x32 = torch.empty(V * 24, dtype=torch.float32, device="cuda")
    capi.amg_random_normal(w["seed"] + 1000, li.STREAM_RHS, 0, V * 12, x)   # a Gaussian field (FP64)
    x32.copy_(x[:V * 24])
    capi.amg_dirac_time(d, x32, 1, capi.AMG_F32, 3, stream=stream)
    ms_d = capi.amg_dirac_time(d, x32, 1, capi.AMG_F32, 10, stream=stream)
    kern["dirac_kernel<P32>"] = {"ms": ms_d, "bytes_per_site": 672, "gb_per_s": 672 * V / (ms_d * 1e-3) / 1e9,
                                 "frac_hbm": 672 * V / (ms_d * 1e-3) / 1e9 / hbm}
    cdims, nc = capi.amg_level_info(h, 1)
    vc = int(np.prod(cdims))
    xc = torch.randn(4 * vc * nc * 2, dtype=torch.float32, device="cuda")
    bf = p.prec_coarsest == capi.AMG_BF16
    capi.amg_coarse_time(h, 1, xc, 1, capi.AMG_F32, 3, stream=stream)
    ms_c = capi.amg_coarse_time(h, 1, xc, 1, capi.AMG_F32, 10, stream=stream)
    cbytes = vc * (9 * nc * nc * (4 if bf else 8) + 2 * nc * 8)
    kern["coarse_apply_kernel<%s>" % ("BF16 operator, FP32 vectors" if bf else "F32")] = {
        "ms": ms_c, "coarse_sites": vc, "nc": nc, "bytes": cbytes, "gb_per_s": cbytes / (ms_c * 1e-3) / 1e9,
        "frac_hbm": cbytes / (ms_c * 1e-3) / 1e9 / hbm}
    if bf:
        # the tensor-core stencil over a lockstep group of four right-hand sides (as the batched coarse
        # solves run it): operand image 2Nc x 9Nc bfloat16 per coarse site + the vectors in and out;
        # useful work 8 * 9 * Nc^2 flop per site and right-hand side against the measured bf16 peak
        bf_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops", 1900.0) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
        capi.amg_coarse_time(h, 1, xc, 4, capi.AMG_BF16, 3, stream=stream)
        ms_t = capi.amg_coarse_time(h, 1, xc, 4, capi.AMG_BF16, 10, stream=stream)
        tbytes = vc * (2 * nc * 9 * nc * 2 + 2 * 4 * nc * 8)
        tflops = 8.0 * 9 * nc * nc * 4 * vc / (ms_t * 1e-3) / 1e12
        kern["coarse_tc_kernel (4 RHS)"] = {"ms": ms_t, "bytes": tbytes, "gb_per_s": tbytes / (ms_t * 1e-3) / 1e9,
                                            "frac_hbm": tbytes / (ms_t * 1e-3) / 1e9 / hbm,
                                            "useful_tflops": tflops, "frac_bf16_peak": tflops / bf_peak}
    del x32, xc
    line = {
        "metric": METRIC, "value": per_rhs, "unit": "ms/RHS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f16+f64", "data": "synthetic", "config": config,
        "roofline": {"kernel": ("sap_half_eo_kernel<P32> (fused SAP half sweep, even-odd domain solves)"
                               if p.sap_eo else SAP_KERNEL_NAMES.get(args.sap_variant, "sap_half (autotuned)")),
                     "bound": "alu",
                     "achieved": sap_tflops, "peak": peak, "unit": "TFLOP/s", "frac": sap_tflops / peak,
                     "traffic": sap_traffic, "rhs_per_launch": width,
                     "peak_kind": f"FP32 FMA from unit counts: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz",
                     "flop_per_step": flop_step, "smoother_ms_per_step": smooth_ms},
        "kernels": kern,
        "e2e": {"value": e2e_ms, "unit": "ms/RHS", "solution_max_rel_diff_vs_device": e2e_diff,
                "batch_width": max(int(i["batch_width"]) for i in e2e_infos),
                "ms_per_step_host_clock": [float(i["ms_total"]) for i in e2e_infos],
                "phase_ms_per_step": {k: float(np.mean([i[k] for i in e2e_infos]))
                                      for k in ("ms_coarse", "ms_smoother", "ms_restrict_prolong", "ms_other",
                                                "ms_products", "ms_orthogonalisation", "ms_true_residual")},
                "h2d_bytes_per_step": int(b.numel() * 8),
                "d2h_bytes_per_step": int(x.numel() * 8)},
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "details": {"volume": V, "setup_ms": setup_ms, "input_generation_s": gen_s, "converged": ok,
                    "outer_iters": float(np.mean([i["iters"] for i in infos])), "cycles": cycles,
                    "true_rel_residual_max": float(max(i["true_rel_residual"] for i in infos)),
                    "phase_ms_per_step": {k: float(np.mean([i[k] for i in infos])) for k in
                                          ("ms_coarse", "ms_smoother", "ms_restrict_prolong", "ms_other",
                                           "ms_products", "ms_orthogonalisation", "ms_true_residual")},
                    "coarse_cycles": float(np.mean([i["coarse_cycles"] for i in infos])),
                    "hbm_peak_gbs": hbm, "hbm_peak_kind": kind, "e2e_steps": ne2e},
    }
    if pool is not None:
        nsamp = pool.procs
        pool.run(pool.procs)                   # warm: every worker has built its sample
        wall = pool.run(nsamp, first=pool.procs)
        pool.close()
        line["cpu_baseline"] = {"value": oracle_extrapolation(wall, nsamp, cycles), "unit": "ms/RHS",
                                "cores": pool.procs, "kind": "oracle",
                                "sample": _sample_text(pool.procs, nsamp, cycles, "this run's GPU solve")}
    capi.amg_hierarchy_destroy(h)
    capi.amg_dirac_destroy(d)
    capi.amg_gauge_destroy(g)
    capi.amg_lattice_destroy(lat)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _setup_field(capi, dims, eps, seed, kappa, csw):
    U = li.gauge_field(dims, eps, seed)
    lat = capi.amg_lattice_create(dims, True)
    g = capi.amg_gauge_create(lat, li.to_interleaved(U))
    d = capi.amg_dirac_create(g, kappa, csw)
    return U, lat, g, d




def run_learned(args):
    """Learned preconditioner on 24^3x48 (exp(0.6iH), seed 5, kappa 0.130):
    train the 1-4-1 parallel-transport network on 4096 (residual, error)
    pairs from the solver (e = (1 - M D) e0, r = D e; amg_learned_train,
    batches of 16), then solve 16 fresh Gaussian right-hand sides (seeds 4000-4015) with
    and without it, and with the same method all in FP64."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi
    dims = (24, 24, 24, 48)
    V = int(np.prod(dims))
    U, lat, g, d = _setup_field(capi, dims, 0.6, 5, 0.130, 1.0)
    p = capi.amg_params_default()
    p.nvec[0] = 24
    v0 = li.to_interleaved(li.test_vectors(dims, 5, 24))
    h = capi.amg_setup(d, p, [v0])
    channels = [1, 4, 1]
    sizes = [channels[l + 1] * channels[l] * 9 * 16 for l in range(2)]
    w = li.to_interleaved(li.complex_normal(5, li.STREAM_NN, (sum(sizes),)) * 0.02).astype(np.float32).reshape(-1)
    W1 = np.zeros((4, 1, 9, 4, 4, 2), np.float32)
    W2 = np.zeros((1, 4, 9, 4, 4, 2), np.float32)
    for a in range(4):
        W1[a, 0, 0, range(4), range(4), 0] = 0.5
        W2[0, a, 0, range(4), range(4), 0] = 0.5
    nn = capi.amg_nn_create(d, channels, w + np.concatenate([W1.reshape(-1), W2.reshape(-1)]))
    npairs, batch = args.pairs, 16
    tp = capi.amg_train_params_default()
    tp.npairs, tp.batch, tp.lr, tp.seed = npairs, batch, 1e-3, 5
    t0 = time.perf_counter()
    losses = list(capi.amg_learned_train(h, nn, tp))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    res = {}
    modes = [("plain", h), ("learned", h)]
    if not args.no_fp64_compare:
        # the same method all in FP64 (smoother, coarse operator and solve), same initial test vectors
        p64 = capi.amg_params_default()
        p64.nvec[0] = 24
        p64.prec_smoother = p64.prec_coarsest = capi.AMG_F64
        t0 = time.perf_counter()
        h64 = capi.amg_setup(d, p64, [v0])
        torch.cuda.synchronize()
        res["fp64_setup_s"] = time.perf_counter() - t0
        modes.append(("plain_fp64", h64))
    for mode, hh in modes:
        if mode != "plain_fp64":
            capi.amg_hierarchy_set_nn(hh, nn if mode == "learned" else None)
        its, ms_l, rel = [], [], []
        for k in range(16):
            bb = torch.from_numpy(li.to_interleaved(li.rhs(dims, 5000 + k - 1000)).reshape(-1)).cuda()
            x = torch.zeros_like(bb)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            st, info = capi.amg_solve(hh, bb, x, 1, TOL, 300)
            ev1.record()
            torch.cuda.synchronize()
            its.append(info.iters)
            ms_l.append(ev0.elapsed_time(ev1))
            rel.append(info.true_rel_residual)
        res[mode] = {"ms_per_rhs": float(np.mean(ms_l)), "outer_iters": float(np.mean(its)),
                     "max_true_rel_residual": float(np.max(rel)), "fallbacks": int(info.nn_fallback)}
        if mode == "plain_fp64":
            capi.amg_hierarchy_destroy(hh)
    line = {"metric": METRIC, "value": res["learned"]["ms_per_rhs"], "unit": "ms/RHS", "n_gpus": 1, "steps": 16,
            "warmup": 0, "ms_per_step": res["learned"]["ms_per_rhs"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights + f32 + f64", "data": "synthetic",
            "config": {"workload": "24^3x48 Wilson-clover (exp(0.6iH), seed 5, kappa 0.130, csw 1.0), 2-level AMG "
                                   "4^4 / 24 test vectors + 1-4-1 PT-conv network",
                       "pairs": npairs, "train_s": train_s, "loss_first": losses[0], "loss_last": losses[-1],
                       "plain": res["plain"], "learned": res["learned"],
                       "plain_fp64": res.get("plain_fp64"), "fp64_setup_s": res.get("fp64_setup_s")}}
    print(json.dumps(line), flush=True)


def run_dirac(args):
    """The Wilson-clover stencil alone (Eq. 1) on 32^3x64 (links exp(0.6iH),
    seed 3, kappa 0.130, c_sw 1.0): mean kernel time per application in FP64,
    FP32 and FP16, against the HBM roofline.  Compulsory bytes per site: input
    and output spinor, the site's four links (each link is read by both of its
    end points, once from HBM) and the clover term.  FP32: 96 + 96 + 4 x 48
    (two-row links) + 288 = 672 B; FP16: 52 + 52 + 4 x 24 + 144 = 344 B
    (per-site scale included); FP64: 192 + 192 + 4 x 144 + 576 = 1536 B."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi
    dims = (32, 32, 32, 64)
    V = int(np.prod(dims))
    t0 = time.perf_counter()
    U, lat, g, d = _setup_field(capi, dims, 0.6, 3, 0.130, 1.0)
    del U
    gen_s = time.perf_counter() - t0
    psi = li.to_interleaved(li.rhs(dims, 3)).reshape(-1)
    hbm, kind = _peaks()
    stream = torch.cuda.current_stream()
    per = {}
    # f64x: float input, FP64 output, links / clover as float hi/lo pairs (full 3x3: 4 x 144 B);
    # f64d: the same arithmetic on FP64 input (every value split into a float pair)
    bytes_site = {"f64": 1536, "f32": 672, "f16": 344, "f64x": 96 + 192 + 4 * 144 + 576,
                  "f64d": 192 + 192 + 4 * 144 + 576}
    # the launch shapes the autotuner picks on this lattice (CTA size, grid cap, register budget)
    shapes = {name: capi.amg_dirac_tune(d, prec)
              for name, prec in (("f64", capi.AMG_F64), ("f32", capi.AMG_F32), ("f16", capi.AMG_F16))}
    with ClockSampler() as clk:
        for name, prec in (("f64", capi.AMG_F64), ("f32", capi.AMG_F32), ("f16", capi.AMG_F16),
                           ("f64x", capi.AMG_F64X), ("f64d", capi.AMG_F64D)):
            x = torch.from_numpy(psi).to(torch.float64 if name in ("f64", "f64d") else torch.float32).cuda()
            capi.amg_dirac_time(d, x, 1, prec, args.warmup, stream=stream)          # warm-up launches
            l0 = capi.amg_launch_count()
            ms = capi.amg_dirac_time(d, x, 1, prec, args.steps, stream=stream)
            launches = capi.amg_launch_count() - l0
            gbs = bytes_site[name] * V / (ms * 1e-3) / 1e9
            per[name] = {"ms_per_apply": ms, "gb_per_s": gbs, "frac_hbm": gbs / hbm, "bytes_per_site": bytes_site[name],
                         "gflops": 1872 * V / (ms * 1e-3) / 1e9, "launches": launches}
            if name in shapes:
                per[name]["launch_shape"] = dict(zip(("threads", "ctas_per_sm_cap", "regs_ctas_per_sm"),
                                                     shapes[name]))
    f32 = per["f32"]
    line = {"metric": "Wilson-clover D application, kernel time (HBM roofline)", "value": f32["ms_per_apply"],
            "unit": "ms/apply", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": f32["ms_per_apply"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "32^3x64 Wilson-clover D (exp(0.6iH) links, seed 3, kappa 0.130, csw 1.0), "
                                   "1 Gaussian field, internal layout", "volume": V,
                       "l2": "working set > L2 (no flush)", "field_generation_s": gen_s, "per_precision": per},
            "roofline": {"kernel": "dirac_kernel<P32>", "bound": "hbm", "achieved": f32["gb_per_s"], "peak": hbm,
                         "unit": "GB/s", "frac": f32["frac_hbm"], "traffic": None, "peak_kind": kind},
            "gpu_launches": per["f32"]["launches"], "clocks": clk.summary()}
    capi.amg_dirac_destroy(d)
    capi.amg_gauge_destroy(g)
    capi.amg_lattice_destroy(lat)
    print(json.dumps(line), flush=True)


def run_mixed3(args):
    """Three grids on 32^3x64 (links exp(0.6iH), seed 3, kappa 0.130, c_sw
    1.0): 4^4 blocks / 24 test vectors, then 2^4 blocks / 32 test vectors;
    FP16 fine smoother with per-site scale, bfloat16 level-1 stencil,
    FGMRES(8) to 1e-1 on level 1, BiCGStab(2) to 1e-2 in FP64 on level 2,
    FP64 outer flexible GMRES(16).  Fresh Gaussian right-hand sides; the same
    hierarchy built all in FP64 is timed on the same right-hand sides."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi
    dims = (32, 32, 32, 64)
    V = int(np.prod(dims))
    t0 = time.perf_counter()
    U, lat, g, d = _setup_field(capi, dims, 0.6, 3, 0.130, 1.0)
    del U
    gen_s = time.perf_counter() - t0
    blocks, nvec = [(4, 4, 4, 4), (2, 2, 2, 2)], [24, 32]
    cdims1 = tuple(dims[mu] // blocks[0][mu] for mu in range(4))
    init = [li.to_interleaved(li.test_vectors(dims, 3, nvec[0])),
            li.to_interleaved(li.coarse_test_vectors(cdims1, 3, nvec[1], 2 * nvec[0]))]
    nsolve = max(1, min(args.steps, 8))
    B = [torch.from_numpy(li.to_interleaved(li.rhs(dims, 3, index=k)).reshape(-1)).cuda() for k in range(nsolve + 1)]
    X = torch.zeros_like(B[0])
    stream = torch.cuda.current_stream()
    res = {}
    variants = [("mixed", capi.AMG_F16, capi.AMG_BF16, capi.AMG_F64)]
    if not args.no_fp64_compare:
        variants.append(("fp64", capi.AMG_F64, capi.AMG_F64, capi.AMG_F64))
    clk_summary = None
    gpu_launches = None
    for name, ps, pc, pcc in variants:
        p = capi.amg_params_default()
        p.nlevels = 3
        for l in range(2):
            for mu in range(4):
                p.block[l][mu] = blocks[l][mu]
            p.nvec[l] = nvec[l]
        p.prec_smoother, p.prec_coarse, p.prec_coarsest = ps, pc, pcc
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = capi.amg_setup(d, p, init)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        X.zero_()
        capi.amg_solve(h, B[nsolve], X, 1, TOL, 500, stream=stream)   # warm-up
        infos = []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler() as clk:
            l0 = capi.amg_launch_count()
            e0.record(stream)
            for k in range(nsolve):
                X.zero_()
                st, info = capi.amg_solve(h, B[k], X, 1, TOL, 500, stream=stream)
                infos.append(info.as_dict())
            e1.record(stream)
            launches = capi.amg_launch_count() - l0
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsolve
        res[name] = {"ms_per_rhs": ms, "setup_ms": setup_ms,
                     "outer_iters": float(np.mean([i["iters"] for i in infos])),
                     "max_true_rel_residual": float(max(i["true_rel_residual"] for i in infos)),
                     "converged": all(i["converged"] == 1 for i in infos),
                     "phase_ms": {k: float(np.mean([i[k] for i in infos])) for k in
                                  ("ms_coarse", "ms_smoother", "ms_restrict_prolong", "ms_other")}}
        if name == "mixed":
            clk_summary, gpu_launches = clk.summary(), launches
        capi.amg_hierarchy_destroy(h)
    line = {"metric": METRIC, "value": res["mixed"]["ms_per_rhs"], "unit": "ms/RHS", "n_gpus": 1, "steps": nsolve,
            "warmup": 1, "ms_per_step": res["mixed"]["ms_per_rhs"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16+bf16+f32+f64", "data": "synthetic",
            "config": {"workload": "32^3x64 Wilson-clover (exp(0.6iH) links, seed 3, kappa 0.130, csw 1.0), "
                                   "3-level AMG 4^4/24 then 2^4/32, FP16 smoother, BF16 level-1 stencil, "
                                   "FGMRES(8) level 1, FP64 BiCGStab(2) level 2, FP64 outer FGMRES(16)",
                       "volume": V, "field_generation_s": gen_s, "l2": "working set > L2 (no flush)",
                       "variants": res},
            "gpu_launches": gpu_launches, "clocks": clk_summary}
    capi.amg_dirac_destroy(d)
    capi.amg_gauge_destroy(g)
    capi.amg_lattice_destroy(lat)
    print(json.dumps(line), flush=True)


def _ragged_pool(capi, hs, warm_b, B, stream):
    """The ragged batch on the stream pool with per-problem step graphs."""
    import torch
    capi.amg_set_ragged_fusion(False)
    try:
        capi.amg_solve_ragged(hs, warm_b, [torch.zeros_like(b) for b in warm_b], TOL, 300)   # captures the graphs
        Xp = [torch.zeros_like(b) for b in B]
        torch.cuda.synchronize()
        l0 = capi.amg_launch_count()
        t0 = time.perf_counter()
        st, infos = capi.amg_solve_ragged(hs, B, Xp, TOL, 300, stream=stream)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3, capi.amg_launch_count() - l0, infos
    finally:
        capi.amg_set_ragged_fusion(True)


def _ragged_sequential(capi, hs, B, X, stream):
    """The batch's solves issued one after another through amg_solve."""
    import torch
    for x in X:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok = []
    for h, b, x in zip(hs, B, X):
        st, info = capi.amg_solve(h, b, x, 1, TOL, 300, stream=stream)
        ok.append(info.converged == 1 and info.true_rel_residual <= TOL)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3, ok


def _ragged_fp64(capi, shapes, probs, init, B, stream, ragged_ms_per_rhs):
    """The plain method all in FP64 on two problems of each size, one after another."""
    import torch
    sample = list(range(6))
    h64 = []
    for i in sample:
        dims, block = shapes[i % 3]
        p = capi.amg_params_default()
        for mu in range(4):
            p.block[0][mu] = block[mu]
        p.nvec[0] = 24
        p.prec_smoother = p.prec_coarsest = capi.AMG_F64
        h64.append(capi.amg_setup(probs[i][3], p, [init[dims]]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok64 = []
    for i, hh in zip(sample, h64):
        x = torch.zeros_like(B[i])
        st, info = capi.amg_solve(hh, B[i], x, 1, TOL, 300, stream=stream)
        ok64.append(info.converged == 1 and info.true_rel_residual <= TOL)
    torch.cuda.synchronize()
    ms64 = (time.perf_counter() - t0) * 1e3
    for hh in h64:
        capi.amg_hierarchy_destroy(hh)
    return {"problems": sample, "ms_per_rhs": ms64 / len(sample), "converged": all(ok64),
            "ragged_ms_per_rhs_same_mix": ragged_ms_per_rhs}


def run_ragged(args):
    """Ragged batch: 64 independent single-RHS solves, problem i (gauge seed
    100 + i) on 8^4 (4^4 blocks), 12^4 (3^4 blocks) or 16^3x32 (4^4 blocks)
    for i % 3 = 0, 1, 2; links exp(0.6iH), kappa 0.130, c_sw 1.0, 24 test
    vectors, FP32 smoother.  The initial test vectors are drawn once per
    lattice size.  One amg_solve_ragged call in its fused form (one launch
    per phase of an Arnoldi step over per-problem descriptors; a warm-up call
    on other right-hand sides first) against the same batch on the stream
    pool with per-problem step graphs, and the same 64 solves issued one
    after another through amg_solve."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi
    shapes = [((8, 8, 8, 8), (4, 4, 4, 4)), ((12, 12, 12, 12), (3, 3, 3, 3)), ((16, 16, 16, 32), (4, 4, 4, 4))]
    n = 64
    init = {dims: li.to_interleaved(li.test_vectors(dims, 100 + k, 24)) for k, (dims, _) in enumerate(shapes)}
    probs = []
    t0 = time.perf_counter()
    for i in range(n):
        dims, block = shapes[i % 3]
        U, lat, g, d = _setup_field(capi, dims, 0.6, 100 + i, 0.130, 1.0)
        p = capi.amg_params_default()
        for mu in range(4):
            p.block[0][mu] = block[mu]
        p.nvec[0] = 24
        h = capi.amg_setup(d, p, [init[dims]])
        probs.append((dims, lat, g, d, h))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    sites = sum(int(np.prod(pr[0])) for pr in probs)

    def rhs_set(base):
        return [torch.from_numpy(li.to_interleaved(li.rhs(pr[0], base + i)).reshape(-1)).cuda()
                for i, pr in enumerate(probs)]
    hs = [pr[4] for pr in probs]
    warm_b = rhs_set(7000)
    capi.amg_solve_ragged(hs, warm_b, [torch.zeros_like(b) for b in warm_b], TOL, 300)
    B = rhs_set(8000)
    X = [torch.zeros_like(b) for b in B]
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    with ClockSampler() as clk:
        l0 = capi.amg_launch_count()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")
        st, infos = capi.amg_solve_ragged(hs, B, X, TOL, 300, stream=stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ragged_ms = (time.perf_counter() - t0) * 1e3
        launches = capi.amg_launch_count() - l0
    ok = all(i.converged == 1 and i.true_rel_residual <= TOL for i in infos)
    # the same batch on the stream pool with per-problem step graphs (the unfused form)
    pool_ms, pool_launches, infos_pool = None, None, []
    if not args.fused_only:
        pool_ms, pool_launches, infos_pool = _ragged_pool(capi, hs, warm_b, B, stream)
    # the same solves one after another
    seq_ms, seq = None, []
    if not args.fused_only:
        seq_ms, seq = _ragged_sequential(capi, hs, B, X, stream)
    # the plain method all in FP64 on a sample of the batch (two problems of each size), one after another
    fp64 = None
    if not args.no_fp64_compare and not args.fused_only:
        fp64 = _ragged_fp64(capi, shapes, probs, init, B, stream, ragged_ms / n)
    line = {"metric": METRIC, "value": ragged_ms / n, "unit": "ms/RHS", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": ragged_ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "ragged batch of 64 single-RHS solves on 8^4 / 12^4 / 16^3x32 (gauge seeds "
                                   "100-163, exp(0.6iH), kappa 0.130, csw 1.0), 2-level AMG, 24 test vectors, "
                                   "FP32 smoother, lockstep FGMRES(16), one launch per phase over per-problem "
                                   "descriptors",
                       "problems": n, "total_sites": sites, "setup_s": setup_s, "converged": ok,
                       "ragged_ms": ragged_ms, "sequential_ms": seq_ms, "sequential_converged": all(seq),
                       "stream_pool_ms": pool_ms, "stream_pool_launches": pool_launches,
                       "stream_pool_converged": all(i.converged == 1 for i in infos_pool),
                       "speedup_vs_stream_pool": pool_ms / ragged_ms if pool_ms else None,
                       "speedup_vs_sequential": seq_ms / ragged_ms if seq_ms else None,
                       "plain_fp64_sequential_sample": fp64,
                       "outer_iters": [int(i.iters) for i in infos]},
            "gpu_launches": launches, "clocks": clk.summary()}
    for dims, lat, g, d, h in probs:
        capi.amg_hierarchy_destroy(h)
        capi.amg_dirac_destroy(d)
        capi.amg_gauge_destroy(g)
        capi.amg_lattice_destroy(lat)
    print(json.dumps(line), flush=True)


def run_coarse_tc(args):
    """The coarse 9-point stencil alone on an 8^3x16 coarse lattice with
    Nc = 48 (16^3x32 fine lattice, links exp(0.6iH), seed 2, kappa 0.130,
    c_sw 1.0, 2^4 blocks, 24 test vectors), stencil stored in bfloat16:
    the tensor-core path (bfloat16 operands, FP32 accumulation, 16 and 8
    right-hand sides per launch) against the SIMT path (FP32 vectors).
    Compulsory bytes per tensor-core launch: the operand image of the stencil
    (2 Nc x 9 Nc bfloat16 per coarse site, 83 KB) plus the nrhs input and
    output vectors (Nc FP32 complex per site each)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi
    dims = (16, 16, 16, 32)
    U, lat, g, d = _setup_field(capi, dims, 0.6, 2, 0.130, 1.0)
    del U
    p = capi.amg_params_default()
    for mu in range(4):
        p.block[0][mu] = 2
    p.nvec[0] = 24
    p.prec_coarsest = capi.AMG_BF16
    h = capi.amg_setup_from_vectors(d, p, [li.to_interleaved(li.test_vectors(dims, 2, 24))])
    cdims, nc = capi.amg_level_info(h, 1)
    Vc = int(np.prod(cdims))
    hbm, kind = _peaks()
    x = li.complex_normal(5, li.STREAM_MISC, (16, Vc, nc))
    xd = torch.from_numpy(li.to_interleaved(x).reshape(-1)).float().cuda()
    stream = torch.cuda.current_stream()
    img_bytes = Vc * 2 * nc * 9 * nc * 2
    res = {}
    with ClockSampler() as clk:
        for name, prec, nrhs in (("tc16", capi.AMG_BF16, 16), ("tc8", capi.AMG_BF16, 8),
                                 ("simt16", capi.AMG_F32, 16), ("simt1", capi.AMG_F32, 1)):
            capi.amg_coarse_time(h, 1, xd, nrhs, prec, args.warmup, stream=stream)
            l0 = capi.amg_launch_count()
            ms = capi.amg_coarse_time(h, 1, xd, nrhs, prec, args.steps, stream=stream)
            launches = capi.amg_launch_count() - l0
            op_bytes = img_bytes if prec == capi.AMG_BF16 else Vc * 9 * nc * nc * 4
            byts = op_bytes + 2 * nrhs * Vc * nc * 8
            flops = 8.0 * 9 * nc * nc * nrhs * Vc
            res[name] = {"nrhs": nrhs, "ms_per_launch": ms, "us_per_rhs": ms * 1e3 / nrhs,
                         "gb_per_s": byts / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm,
                         "useful_tflops": flops / (ms * 1e-3) / 1e12, "bytes_per_launch": byts,
                         "launches": launches}
    t = res["tc16"]
    line = {"metric": "coarse 9-point stencil, kernel time per right-hand side (HBM roofline)",
            "value": t["us_per_rhs"], "unit": "us/RHS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t["ms_per_launch"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 operands, f32 accumulate", "data": "synthetic",
            "config": {"workload": "coarse stencil, 8^3x16 coarse sites x Nc 48 (16^3x32 fine, 2^4 blocks, 24 test "
                                   "vectors), bfloat16 stencil, 16 right-hand sides per tensor-core launch",
                       "coarse_sites": Vc, "nc": nc, "l2": "operator image 680 MB > L2 (no flush)",
                       "variants": res},
            # traffic: dram__bytes_read.sum + dram__bytes_write.sum of one coarse_tc_kernel<32> launch (16 RHS)
            # on this workload from an ncu --set full capture (708.8 + 47.6 MB)
            "roofline": {"kernel": "coarse_tc_kernel<32>", "bound": "hbm", "achieved": t["gb_per_s"], "peak": hbm,
                         "unit": "GB/s", "frac": t["frac_hbm"], "traffic": 756.4e6, "peak_kind": kind},
            "gpu_launches": t["launches"], "clocks": clk.summary()}
    capi.amg_hierarchy_destroy(h)
    capi.amg_dirac_destroy(d)
    capi.amg_gauge_destroy(g)
    capi.amg_lattice_destroy(lat)
    print(json.dumps(line), flush=True)


def run_solve16(args):
    """One complex Gaussian source per step on 16^3 x 32 (links exp(0.6iH), seed 2,
    kappa 0.130, c_sw 1.0), 2-level AMG 4^4 / 24 test vectors, FGMRES(16) FP64 outer;
    the round-trip end-to-end leg copies each step's source and solution."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi

    w = SOLVE16
    dims = w["dims"]
    V = int(np.prod(dims))
    prec = {"f64": capi.AMG_F64, "f32": capi.AMG_F32, "f16": capi.AMG_F16}[args.prec]
    U = li.gauge_field(dims, w["eps"], w["seed"])
    lat = capi.amg_lattice_create(dims, True)
    g = capi.amg_gauge_create(lat, li.to_interleaved(U))
    d = capi.amg_dirac_create(g, w["kappa"], w["csw"])
    v0 = li.to_interleaved(li.test_vectors(dims, w["seed"], w["nvec"]))
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    setup_kw = {"n_init": args.n_init, "n_adapt": args.n_adapt, "coarse_tol": args.coarse_tol}
    h = capi.amg_setup(d, make_params(capi, prec, args.coarse_prec, args.outer, args.sap_variant, setup_kw,
                                      args.vec_prec, w=w), [v0])
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3

    nsteps = args.warmup + args.steps
    # right-hand sides: one per step and rank, resident in HBM before timing
    B = [torch.from_numpy(li.to_interleaved(li.rhs(dims, w["seed"], index=rank * nsteps + k)).reshape(-1)).cuda()
         for k in range(nsteps)]
    X = torch.zeros_like(B[0])
    infos = []
    for k in range(args.warmup):
        X.zero_()
        capi.amg_solve(h, B[k], X, 1, TOL, 500, stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler() as clk:
        torch.cuda.nvtx.range_push("timed")
        launches0 = capi.amg_launch_count()
        ev0.record(stream)
        for k in range(args.warmup, nsteps):
            X.zero_()
            st, info = capi.amg_solve(h, B[k], X, 1, TOL, 500, stream=stream)
            infos.append(info.as_dict())
        ev1.record(stream)
        gpu_launches = capi.amg_launch_count() - launches0
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    per_rhs = ms / (args.steps * world)
    ok = all(i["converged"] == 1 and i["true_rel_residual"] <= TOL for i in infos)

    # end-to-end through the public API with host buffers (pinned), copies timed
    hb = [B[k].cpu().pin_memory() for k in range(args.warmup, nsteps)]
    hx = torch.empty_like(hb[0]).pin_memory()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        bd = hb[k].to("cuda", non_blocking=True)
        X.zero_()
        capi.amg_solve(h, bd, X, 1, TOL, 500, stream=stream)
        hx.copy_(X, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    # Roofline of the dominant kernel of the solve, the fused SAP half sweep
    # (one launch = one colour of domains).  Average launch duration from the
    # library's CUDA-event smoother timer: 2 * sap_iters launches per cycle.
    # Algorithmic work per active site (standard Wilson-clover count, 1872
    # flop per site for D): residual b - D x (1872 + 24) + 6 minimal-residual
    # steps on D_SAP (1494 for the in-domain hops and clover of a 4^4 domain,
    # + 336 for the two dot products and two updates) = 12876 flop; half the
    # sites are active per launch.  12.8 flop/byte puts it on the ALU side of
    # the ridge, so it is reported against the FP32 FMA peak:
    # 152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s (nominal).
    p = make_params(capi, prec, args.coarse_prec, args.outer, args.sap_variant, setup_kw, args.vec_prec, w=w)
    iters = np.mean([i["iters"] for i in infos])
    smooth_ms = np.mean([i["ms_smoother"] for i in infos])
    cycles = np.mean([i["cycles"] for i in infos])
    launches = 2 * p.sap_iters * cycles
    sap_launch_us = smooth_ms / launches * 1e3
    flop_site = 1872 + 24 + p.mr_iters * (1494 + 336)
    flop_launch = flop_site * V / 2
    achieved = flop_launch / (sap_launch_us * 1e-6) / 1e12
    peak, sms, mhz = _fp32_fma_peak(torch)
    hbm_peak, peak_kind = _peaks()

    line = {
        "metric": METRIC, "value": per_rhs, "unit": "ms/RHS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32+f64", "f16": "f16+f32+f64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": "16^3x32 Wilson-clover (exp(0.6iH) links, seed 2, kappa 0.130, csw 1.0), "
                               "2-level AMG 4^4 blocks, 24 test vectors, SAP(4) x MR(6), BiCGStab(2) coarse to 1e-2, "
                               "FGMRES(16) FP64 outer, 1 Gaussian RHS per step",
                   "smoother_prec": args.prec, "coarse_prec": args.coarse_prec, "vector_prec": args.vec_prec,
                   "outer_solver": args.outer,
                   "n_init": p.n_init, "n_adapt": p.n_adapt, "coarse_tol": p.coarse_tol,
                   "setup_ms": setup_ms, "l2": "working set > L2 (no flush)",
                   "outer_iters": float(iters), "cycles": float(cycles), "converged": ok,
                   "phase_ms": {k: float(np.mean([i[k] for i in infos])) for k in
                                ("ms_coarse", "ms_smoother", "ms_restrict_prolong", "ms_other", "ms_products",
                                 "ms_orthogonalisation", "ms_true_residual")},
                   "coarse_cycles": float(np.mean([i["coarse_cycles"] for i in infos]))},
        # traffic: the per-site DRAM count of the current kernel's capture (24^3x48, 12 right-hand
        # sides per launch) scaled to this workload's launches (one right-hand side); variant 0 only
        "roofline": {"kernel": SAP_KERNEL_NAMES.get(args.sap_variant, "sap_half (autotuned)"),
                     "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (SAP_DRAM_BYTES_PER_SITE_RHS * V / 2
                                 if (args.sap_variant == 0 and args.prec == "f32") else None),
                     "peak_kind": f"FP32 FMA from unit counts: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz",
                     "avg_launch_us": sap_launch_us, "flop_per_launch": flop_launch,
                     "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": peak_kind},
        "e2e": {"value": e2e_ms, "unit": "ms/RHS", "h2d_bytes_per_step": int(hb[0].numel() * 8),
                "d2h_bytes_per_step": int(hx.numel() * 8)},
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
    }
    if args.outer == "mbicgs":
        # no SAP in this solve: the smoother timer holds the inner BiCGStab(2) on D
        line.pop("roofline")
        line["config"]["workload"] = line["config"]["workload"].replace(
            "2-level AMG 4^4 blocks, 24 test vectors, SAP(4) x MR(6), BiCGStab(2) coarse to 1e-2, FGMRES(16) FP64 outer",
            "MBiCGs: flexible BiCGStab FP64 outer preconditioned by FP32 BiCGStab(2) on D to 1e-4 (no multigrid)")
    capi.amg_hierarchy_destroy(h)
    capi.amg_dirac_destroy(d)
    capi.amg_gauge_destroy(g)
    capi.amg_lattice_destroy(lat)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()




def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="propagator",
                    choices=["propagator", "solve16", "learned", "dirac", "mixed3", "ragged", "coarse_tc"])
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--prop-coarse", default="bf16", choices=["f32", "bf16"],
                    help="propagator: coarsest operator storage (bf16, the default: bfloat16 entries)")
    ap.add_argument("--no-coarse-tc", action="store_true",
                    help="propagator with bf16: batched coarse solves on the SIMT solver instead of the tensor cores")
    ap.add_argument("--resid-pair", action="store_true",
                    help="propagator: the outer solver's true residual in double-float pair arithmetic on the "
                         "FP32 pipe (about 46 significant bits) instead of the FP64 stencil")
    ap.add_argument("--sap-eo", action="store_true",
                    help="propagator: even-odd (Schur complement) SAP domain solves")
    ap.add_argument("--mr", type=int, default=None, help="propagator: minimal-residual steps per domain solve")
    ap.add_argument("--dims", default=None,
                    help="propagator workload on a smaller lattice Lx,Ly,Lz,Lt (profiling; not the headline)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--fused-only", action="store_true",
                    help="ragged workload: time the fused batch only (no stream-pool or one-by-one comparison)")
    ap.add_argument("--sap-variant", type=int, default=0, choices=[-1, 0, 1, 2, 3],
                    help="SAP kernel: 0 operator through L1/L2 (default), 1 staged in shared memory, "
                         "2 two right-hand sides of a batch per CTA, -1 autotune")
    ap.add_argument("--n-init", type=int, default=None, help="setup (0-a) SAP applications (default: library's)")
    ap.add_argument("--n-adapt", type=int, default=None, help="setup (0-b) adaptive passes (default: library's)")
    ap.add_argument("--coarse-tol", type=float, default=None, help="coarsest solve tolerance (default: library's)")
    ap.add_argument("--outer", default="fgmres", choices=["fgmres", "fbicgstab", "mbicgs"],
                    help="outer solver of the solve16 workload (fbicgstab: the paper's flexible BiCGStab; "
                         "mbicgs: the paper's mixed-precision BiCGStab comparison solver, no multigrid)")
    ap.add_argument("--vec-prec", default="f16", choices=["f32", "f16"],
                    help="solve16: test vectors as restriction and prolongation read them (f16: half storage "
                         "with a per-site scale, FP32 arithmetic; f32: the setup's precision)")
    ap.add_argument("--coarse-prec", default="f32", choices=["f32", "bf16"],
                    help="solve16: coarsest stencil storage (bf16: bfloat16 entries, FP32 arithmetic)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return {"propagator": run_headline, "solve16": run_solve16, "learned": run_learned, "dirac": run_dirac,
            "mixed3": run_mixed3, "ragged": run_ragged, "coarse_tc": run_coarse_tc}[args.workload](args)


if __name__ == "__main__":
    main()
