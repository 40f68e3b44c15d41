"""Throughput of the many-chain surrogate mMALA step (proposals/s) on GB300.

One step = one transition of every chain of the workload: reduced proposal,
tensor-core MLP forward and Jacobian, FP64 Gauss-Newton Cholesky and
log-acceptance, complement draw and field update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Default workload: 16384 chains, r = 200 DIS basis, GELU 200-400-400-100,
65 x 65 grid, dt = 0.5, BF16 slices on tcgen05 with FP64 Cholesky.  The FP64
plain step (4096 chains, r = 200 KLE) is timed beside it.  With N > 1 (under
torchrun) every rank runs its own chain shard (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from workloads import (BASIS_KLE, CONFIGS, SEED_CHAINS, make_data,  # noqa: E402
                       surrogate_inputs)

METRIC = "mMALA proposals/s at r=200 (BF16/FP32 vs FP64 plain)"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak of GB300 from the pool's profiling notes (no measured FP64 figure exists)
FP64_NOMINAL_TFLOPS = 1.25
# Ceiling of FP64-accurate work done as double-float arithmetic on the FP32
# pipe: 152 SMs x 128 FP32 lanes x 2.07 GHz FP32 instructions per second,
# 12 of them per double-float multiply-add (the compensated dot-product step
# of the factorisation), 2 flops per multiply-add.
FP32_LANES, SMS, SM_GHZ, DF_INSTR_PER_FMA = 128, 152, 2.07, 12
FP32_PEAK_TFLOPS = SMS * FP32_LANES * SM_GHZ * 1e9 * 2 / 1e12
DF_PEAK_TFLOPS = FP32_PEAK_TFLOPS / DF_INSTR_PER_FMA


def geometry_traffic_per_chain(workload: str):
    """DRAM bytes per chain of the geometry kernel from its committed ncu summary.

    The capture ran the same kernel on a 1216-chain case of the same workload;
    the per-chain traffic does not depend on the chain count.  None when no
    capture of this workload's kernel exists.
    """
    w = CONFIGS[workload]
    kernel = "k_wb_geometry" if w.d_y < w.r else "k_geometry"
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        with open(path) as fh:
            for line in fh:
                if line.strip().startswith("dram_bytes_per_chain:"):
                    return float(line.split(":")[1])
    except OSError:
        pass
    return None


def geometry_work(r: int, d_y: int, tc_gram: bool = False) -> dict:
    """Algorithmic work of one geometry launch per chain, by pipe.

    d_y < r (Woodbury path): in double-float arithmetic the bordered Cholesky
    of the (d_y + 1)-matrix, (d_y + 1)^3 / 3, and unless they were formed
    beforehand (tc_gram: the BF16 path with d_y <= 128, where the tensor cores
    form J J^T and a row-product kernel K b and K a) the FP32 Gram product
    J J^T, d_y (d_y + 1) r flops, and the products K b and K a, 4 r d_y.  Otherwise: the FP32 product J^T J, r (r + 1) d_y, and in
    double-float the bordered r-Cholesky with the reverse-density products and
    the gradient (`fp64_flops_geometry`).  A double-float multiply-add takes 12
    FP32 instructions, so the FP32-pipe charge is fp32 + 12 x df flops.
    """
    if d_y < r:
        fp32 = 0 if tc_gram else d_y * (d_y + 1) * r
        df = (d_y + 1) ** 3 / 3.0 + (0.0 if tc_gram else 4.0 * r * d_y)
    else:
        fp32 = r * (r + 1) * d_y
        df = fp64_flops_geometry(r, d_y)
    return {"fp32": fp32, "df": df, "fp32_charge": fp32 + DF_INSTR_PER_FMA * df}


def load_peaks() -> dict:
    """The measured HBM and bf16 peaks of this GPU pool (empty when absent)."""
    try:
        with open(PEAKS_PATH) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def jacobian_flops(w, slice_products: int = 1) -> float:
    """Flops per chain of the Jacobian GEMMs in the order the library picks
    (Sec. 4.3's min{d_y, r} rule): reverse 2 d_y sum_{l=0}^{L-2} w_l w_{l+1},
    forward 2 r sum_{l=1}^{L-1} w_l w_{l+1}, the smaller (reverse on a tie or
    when d_y < r).  slice_products = 1 gives the algorithmic work, 3 the
    products the default two-slice scheme issues."""
    ws = list(w.widths)
    L = len(ws) - 1
    rev = sum(2.0 * w.d_y * ws[l] * ws[l + 1] for l in range(0, L - 1))
    fwd = sum(2.0 * w.r * ws[l] * ws[l + 1] for l in range(1, L))
    use = fwd if (w.r < w.d_y and fwd < rev) else rev
    return slice_products * use


def tensor_flops_per_proposal(w) -> float:
    """Algorithmic dense-contraction flops of one proposal: MLP forward,
    Jacobian, the Gauss-Newton Gram product (the smaller of J^T J and J J^T)
    and the two complement projections (E M and D coef2)."""
    ws = list(w.widths)
    fwd = sum(2.0 * ws[l] * ws[l + 1] for l in range(len(ws) - 1))
    gram = 2.0 * min(w.r, w.d_y) ** 2 * max(w.r, w.d_y)
    return fwd + jacobian_flops(w) + gram + 2 * 2.0 * w.N * w.r


def fp64_flops_geometry(r: int, d_y: int) -> float:
    """Algorithmic FP64 flops of one geometry launch per chain.

    Cholesky of I + H bordered by one row, (r+1)^3/3; the products L^T b and
    L^T a of the reverse density, 2 r^2; the gradient J^T res, 2 r d_y.  The
    Gauss-Newton product J^T J runs in FP32 and is not counted.
    """
    return (r + 1) ** 3 / 3.0 + 2.0 * r * r + 2.0 * r * d_y


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.result = None
        if self.proc is None:
            return False
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 7]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[4 + k].strip().lower() == "active":
                    reasons.add(nm)
        if sm:
            loaded = [x for x in sm if x > 0.5 * (mx or max(sm))] or sm
            self.result = {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx,
                           "reasons": sorted(reasons), "samples": len(sm)}
        return False


def load_surrogate(dino, ctx, w):
    inp = surrogate_inputs(w)
    prec = dino.DINO_PREC_BF16 if w.precision == "bf16" else dino.DINO_PREC_FP64
    sid = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=w.r,
        widths=w.widths, activation=w.activation, W=inp["Ws"], b=inp["bs"],
        basis_kind=w.basis_kind, basis_gauss=inp["G"], precision=prec,
        noise_map={"auto": 0, "cholesky": 1, "perturbation": 2, "eigen": 3}[w.noise_map])
    twin = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=w.r,
        widths=w.widths, activation=w.activation, W=inp["Ws"], b=inp["bs"],
        basis_kind=BASIS_KLE, precision=dino.DINO_PREC_FP64)
    f0 = dino.dino_surrogate_eval(ctx, twin, inp["m_true_r"], w.d_y, want_L=False)["f"][0]
    dino.dino_unload_surrogate(ctx, twin)
    y, nv = make_data(f0, inp["eps"], w.noise_frac)
    dino.dino_set_data(ctx, sid, y, nv)
    return sid


def shard_base(rank: int, chains_per_rank: int) -> int:
    """Global id of this rank's first chain: ranks own consecutive chain ranges,
    so a chain's random numbers (keyed by its global id) do not depend on N."""
    return rank * chains_per_rank


def timed_repeats(dino, ctx, pool, steps, st, barrier, repeats):
    """Device times of `repeats` passes of `steps` transitions; the median pass."""
    times = [timed_steps(dino, ctx, pool, steps, st, barrier) for _ in range(repeats)]
    return statistics.median(times), times


def timed_steps(dino, ctx, pool, steps, st, barrier):
    """Device time of `steps` transitions (CUDA events on the stream the library launches on)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    dino.dino_chains_step(ctx, pool, steps, stats=False)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / 1e3


def run_ours(args, rank, world, device):
    import torch
    import paper_2403_08220_gb300 as dino

    torch.cuda.set_device(device)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", device))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    w = CONFIGS[args.workload]
    C = args.chains or w.n_chains
    # a dedicated stream: the library launches every kernel on it and the
    # CUDA events below are recorded on it
    stream = torch.cuda.Stream(device=device)
    assert stream.cuda_stream != 0
    ctx = dino.dino_init(device, 0, stream.cuda_stream, 0)
    fp32_peak = dino.dino_measure_fp32_peak(ctx)
    sid = load_surrogate(dino, ctx, w)
    info = dino.dino_surrogate_query(ctx, sid)
    base = shard_base(rank, C)            # weak scaling: each rank owns its chain range
    pool = dino.dino_chains_create(ctx, sid, C, w.dt, SEED_CHAINS, base)
    dino.dino_chains_step(ctx, pool, args.warmup, stats=False)
    dino.dino_sync(ctx)
    n0 = dino.dino_launch_count(ctx)
    with ClockSampler(device) as clk:
        secs, rep_secs = timed_repeats(dino, ctx, pool, args.steps, stream, barrier, args.repeats)
    launches = (dino.dino_launch_count(ctx) - n0) // args.repeats
    stats = dino.dino_chains_step(ctx, pool, 1)
    secs = max_over_ranks(secs)
    value = world * C * args.steps / secs

    # per-kernel times (CUDA events around each launch) over a second pass
    ctx_t = dino.dino_init(device, 0, stream.cuda_stream, dino.DINO_FLAG_TIMING)
    sid_t = load_surrogate(dino, ctx_t, w)
    pool_t = dino.dino_chains_create(ctx_t, sid_t, C, w.dt, SEED_CHAINS, base)
    dino.dino_chains_step(ctx_t, pool_t, 1, stats=False)
    dino.dino_kernel_times(ctx_t, reset=True)
    n_pass = max(2, min(args.steps, 5))
    dino.dino_chains_step(ctx_t, pool_t, n_pass, stats=False)
    kt = dino.dino_kernel_times(ctx_t)
    dino.dino_chains_destroy(ctx_t, pool_t)
    ctx_t.close()
    total = sum(v[0] for v in kt.values()) or 1.0
    geo = kt.get("geometry", max(kt.values(), key=lambda v: v[0]))
    geo_ms = geo[0] / max(1, geo[1])
    tc_gram = bool(info["gram_on_tensor_cores"])
    work = geometry_work(w.r, w.d_y, tc_gram)
    achieved = work["fp32_charge"] * C / (geo_ms * 1e-3) / 1e12
    tpc = geometry_traffic_per_chain(args.workload)
    roofline = {"bound": "alu", "pipe": "fp32", "kernel": "geometry",
                "achieved": round(achieved, 4), "peak": round(fp32_peak, 2),
                "peak_source": "measured: dino_measure_fp32_peak (independent FMA chains on "
                               "every SM, CUDA events); double-float multiply-adds charged at "
                               "12 FP32 instructions",
                "unit": "TFLOP/s", "frac": round(achieved / fp32_peak, 4),
                "work_per_chain": {"fp32_flops": work["fp32"], "df_flops": work["df"]},
                "traffic": tpc * C if tpc else None,
                "traffic_note": "dram bytes per launch scaled from a 1216-chain ncu capture",
                "share_of_step": round(geo[0] / total, 4)}
    peaks = load_peaks()
    bf16_sus = peaks.get("bf16_tflops_sustained")
    hbm = peaks.get("hbm_gbs")
    # the largest tensor-core kernel beside it: the Jacobian GEMMs, against
    # the measured sustained bf16 peak; algorithmic flops (one product) and
    # the slice products the default two-slice scheme issues
    roofline_tensor = None
    jt = kt.get("jac_tc")
    if jt and w.precision == "bf16":
        alg = jacobian_flops(w) * C * n_pass / (jt[0] * 1e-3) / 1e12
        iss = jacobian_flops(w, 3) * C * n_pass / (jt[0] * 1e-3) / 1e12
        roofline_tensor = {"bound": "tensor", "kernel": "jac_tc (k_tc_gemm, Jacobian)",
                           "achieved": round(alg, 2), "achieved_issued": round(iss, 2),
                           "peak": bf16_sus, "unit": "TFLOP/s",
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained",
                           "frac": round(alg / bf16_sus, 4) if bf16_sus else None,
                           "frac_issued": round(iss / bf16_sus, 4) if bf16_sus else None,
                           "flops_per_chain": jacobian_flops(w),
                           "flops_per_chain_issued": jacobian_flops(w, 3),
                           "share_of_step": round(jt[0] / total, 4)}
    # the whole step against the per-proposal algorithmic work of the hot
    # path (tensor: MLP, Jacobian, Gram, projections; HBM: 249 KB of chain
    # state per proposal at r = 200)
    tpp = tensor_flops_per_proposal(w)
    step_fractions = {
        "tensor_mflop_per_proposal": round(tpp / 1e6, 2),
        "tensor_frac_of_sustained_bf16": round(tpp * value / world / (bf16_sus * 1e12), 4)
        if bf16_sus else None,
        "hbm_kb_per_proposal": 249.0,
        "hbm_frac": round(249e3 * value / world / (hbm * 1e9), 4) if hbm else None}

    # a step size that mixes (prior-draw starts, dt = 2e-5: about a sixth of
    # the proposals accepted), so that the accept path's stores are timed
    mix = None
    if not args.skip_mixing:
        pm = dino.dino_chains_create(ctx, sid, C, 2e-5, SEED_CHAINS, base)
        dino.dino_chains_step(ctx, pm, args.warmup, stats=False)
        sm_, _ = timed_repeats(dino, ctx, pm, args.steps, stream, barrier, 3)
        st_m = dino.dino_chains_step(ctx, pm, args.steps)
        mix = {"dt": 2e-5, "proposals_per_s": world * C * args.steps / max_over_ranks(sm_),
               "ms_per_step": 1e3 * sm_ / args.steps,
               "acceptance_rate": st_m["accepts"] / max(1, st_m["proposals"])}
        dino.dino_chains_destroy(ctx, pm)

    # FP64 plain step beside it (fewer steps: it runs its GEMMs in FP64)
    fp64_line = None
    if not args.skip_fp64 and rank == 0:
        w64 = CONFIGS["r200_kle_fp64"]
        sid64 = load_surrogate(dino, ctx, w64)
        p64 = dino.dino_chains_create(ctx, sid64, w64.n_chains, w64.dt, SEED_CHAINS)
        dino.dino_chains_step(ctx, p64, 1, stats=False)
        k64 = max(1, min(5, args.steps))
        s64 = timed_steps(dino, ctx, p64, k64, stream, lambda: None)
        fp64_line = {"workload": "r200_kle_fp64", "chains": w64.n_chains, "steps": k64,
                     "proposals_per_s": w64.n_chains * k64 / s64,
                     "ms_per_step": 1e3 * s64 / k64}
        dino.dino_chains_destroy(ctx, p64)

    # end to end through the C ABI with host buffers: create from a host m0,
    # run the steps, read the reduced states and misfits back
    e2e = None
    if not args.skip_e2e:
        rng = np.random.default_rng(rank)
        m0 = np.ascontiguousarray(0.05 * rng.standard_normal((C, w.N)))
        barrier()
        t0 = time.perf_counter()
        pe = dino.dino_chains_create(ctx, sid, C, w.dt, SEED_CHAINS, base, m0)
        dino.dino_chains_step(ctx, pe, args.steps, stats=False)
        st = dino.dino_chains_read(ctx, pe, C, w.r, w.N, field=False)
        el = max_over_ranks(time.perf_counter() - t0)
        dino.dino_chains_destroy(ctx, pe)
        e2e = {"value": world * C * args.steps / el, "unit": "proposals/s",
               "h2d_bytes_per_step": int(m0.nbytes / args.steps),
               "d2h_bytes_per_step": int((st["m_r"].nbytes + st["phi"].nbytes +
                                          st["accepts"].nbytes) / args.steps),
               "what": f"create {C} chains from host fields + {args.steps} steps + read m_r, phi"}
    dino.dino_chains_destroy(ctx, pool)
    ctx.close()

    line = None
    if rank == 0:
        slots = state_bytes(w, C, info)
        line = {
            "metric": METRIC, "value": value, "unit": "proposals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 GEMMs (fp32 accumulation) + double-float (fp32 pairs) Cholesky and "
                     "solves + f64 log-ratio",
            "data": "synthetic (seeded weights, DIS basis, data from the surrogate at a seeded truth)",
            "config": {"workload": f"{args.workload}: {C} chains/GPU, r={w.r} "
                                   f"{'DIS' if w.basis_kind else 'KLE'}, MLP "
                                   f"{'-'.join(map(str, w.widths))} GELU, N={w.N}, dt={w.dt}",
                       "l2": "inputs larger than L2 (chain state %.2f GB: %s)"
                             % (slots["total"] / 1e9, slots["what"]),
                       "repeats": f"median of {args.repeats} timed passes of {args.steps} steps",
                       "parallelism": f"chains sharded over {world} GPU(s)"},
            "roofline": roofline, "roofline_tensor": roofline_tensor,
            "step_fractions": step_fractions,
            "gpu_launches": int(launches),
            "acceptance_rate": stats["accepts"] / max(1, stats["proposals"]),
            "repeat_ms_per_step": [round(1e3 * t / args.steps, 4) for t in rep_secs],
            "kernel_share": {k: round(v[0] / total, 4) for k, v in kt.items()},
            "mixing": mix, "fp64_plain": fp64_line, "e2e": e2e,
            "clocks": clk.result,
        }
    if dist is not None:
        dist.destroy_process_group()
    return line


def state_bytes(w, C, info) -> dict:
    """Device bytes of the chain state a step reads: the two factor slots,
    the Jacobian state of the d_y-sized paths and the field."""
    r, dy = w.r, w.d_y
    fe = 4 if w.precision == "bf16" else 8
    if info["noise_map"] == "perturbation":
        slot = ((dy + 1) * (dy + 2) // 2 + (dy + 1) + 2 * dy + 2) * 8
        js = C * dy * r * fe
        what = "perturbation-map factor slots and J state"
    elif info["noise_map"] == "eigen":
        slot = (dy * dy + 3 * dy + 2) * 8
        js = C * dy * r * fe
        what = "eigen-map slots and J state"
    else:
        slot = ((r + 1) * (r + 2) // 2 + r + 1) * 8
        js = 0
        what = "Cholesky factor slots"
    total = 2 * C * slot + js + C * w.N * fe
    return {"total": total, "what": what + " + field"}


def run_hetero(args, device=0):
    """Eight posteriors of different size (r = 32 ... 400) stepped together.

    One step = one transition of every chain of all eight pools, issued by
    dino_chains_step_many, which runs each pool on a stream of its own so
    that their kernels overlap.  The same steps issued pool after pool on one
    stream are timed beside it.
    """
    import torch
    import paper_2403_08220_gb300 as dino
    from workloads import heterogeneous_workloads
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device=device)
    ctx = dino.dino_init(device, 0, stream.cuda_stream, 0)
    fp32_peak = dino.dino_measure_fp32_peak(ctx)
    ws = heterogeneous_workloads()
    if args.hetero_r:  # one posterior of the eight (a small case for a profile)
        ws = [w for w in ws if w.r == args.hetero_r]
        if not ws:
            raise SystemExit(f"no heterogeneous posterior with r = {args.hetero_r}")
    pools, infos = [], []
    for w in ws:
        sid = load_surrogate(dino, ctx, w)
        infos.append(dino.dino_surrogate_query(ctx, sid))
        pools.append(dino.dino_chains_create(ctx, sid, w.n_chains, w.dt, SEED_CHAINS))
    dino.dino_chains_step_many(ctx, pools, 2)
    steps = max(1, min(args.steps, 10))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    conc = statistics.median(timed(lambda: dino.dino_chains_step_many(ctx, pools, steps))
                             for _ in range(3))

    def sequential():
        for _ in range(steps):
            for p in pools:
                dino.dino_chains_step(ctx, p, 1, stats=False)
    seq = timed(sequential)
    total = sum(w.n_chains for w in ws) * steps
    tflops = sum(w.n_chains * tensor_flops_per_proposal(w) for w in ws) * steps / conc / 1e12
    charge = sum(w.n_chains * geometry_work(w.r, w.d_y, bool(i["gram_on_tensor_cores"]))
                 ["fp32_charge"] for w, i in zip(ws, infos)) * steps / conc / 1e12
    peaks = load_peaks()
    bf16_sus = peaks.get("bf16_tflops_sustained")
    for p in pools:
        dino.dino_chains_destroy(ctx, p)
    ctx.close()
    return {"workload": "8 posteriors, r in {32,...,400}, d_y in {50,...,400}, MLP r-2r-2r-d_y "
                        "GELU, 512-8192 chains, N=4225, dt=0.5, stepped concurrently",
            "proposals_per_s": total / conc, "ms_per_step": 1e3 * conc / steps,
            "sequential_ms_per_step": 1e3 * seq / steps,
            "chains": [w.n_chains for w in ws], "r": [w.r for w in ws], "d_y": [w.d_y for w in ws],
            "jacobian_mode": ["forward" if i["jac_forward"] else "reverse" for i in infos],
            "noise_map": [i["noise_map"] for i in infos],
            "roofline": {
                "tensor_achieved_tflops": round(tflops, 2),
                "tensor_frac_of_sustained_bf16": round(tflops / bf16_sus, 4) if bf16_sus else None,
                "fp32_pipe_charge_tflops": round(charge, 2),
                "fp32_frac_of_measured": round(charge / fp32_peak, 4),
                "note": "whole-step rates: algorithmic tensor flops (MLP, Jacobian, Gram, "
                        "projections) and the geometry kernels' FP32-pipe charge over the step time"}}


def library_kle_rows(dino, ctx, w, lo, hi):
    """Rows lo .. hi - 1 of the library's own KLE encoder on w's grid."""
    Ws = [np.zeros((2, hi)), np.zeros((2, 2))]
    sid = dino.dino_load_surrogate(
        ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta, r=hi,
        widths=[hi, 2, 2], activation=1, W=Ws, b=[np.zeros(2), np.zeros(2)],
        basis_kind=BASIS_KLE)
    E, _ = dino.dino_read_basis(ctx, sid, hi, w.N)
    dino.dino_unload_surrogate(ctx, sid)
    return E[lo:hi]


def run_da(args, device=0):
    """Delayed acceptance (Algorithm 1's second stage) on the r = 200 workload.

    True map: the surrogate's network reading 200 further KLE coordinates of
    the field (E_t = [E; KLE rows 200..399], weights from
    workloads.true_model_weights, eps = 0.05).  dt = 2e-5 from prior draws,
    where the first stage accepts about a sixth of the proposals.
    """
    import torch
    import paper_2403_08220_gb300 as dino
    from workloads import true_model_weights
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device=device)
    ctx = dino.dino_init(device, 0, stream.cuda_stream, 0)
    w = CONFIGS["r200_dis_bf16"]
    C, dt = w.n_chains, 2e-5
    out = {"workload": f"r200_dis_bf16 + true map on a 400-dim encoding, {C} chains, dt={dt}"}
    for da in (False, True):
        sid = load_surrogate(dino, ctx, w)
        if da:
            E, _ = dino.dino_read_basis(ctx, sid, w.r, w.N)
            Et = np.vstack([E, library_kle_rows(dino, ctx, w, w.r, 2 * w.r)])
            Wt, bt = true_model_weights(w, w.r, 0.05)
            dino.dino_set_true_model(ctx, sid, E_t=Et, W=Wt, b=bt, activation=w.activation)
        pool = dino.dino_chains_create(ctx, sid, C, dt, SEED_CHAINS)
        dino.dino_chains_step(ctx, pool, 3, stats=False)
        secs, _ = timed_repeats(dino, ctx, pool, args.steps, stream, lambda: None, 3)
        st = dino.dino_chains_step(ctx, pool, args.steps)
        key = "two_stage" if da else "surrogate_only"
        out[key] = {"proposals_per_s": C * args.steps / secs,
                    "ms_per_step": 1e3 * secs / args.steps,
                    "stage1_acceptance": st["stage1_accepts"] / max(1, st["proposals"]),
                    "acceptance": st["accepts"] / max(1, st["proposals"])}
        dino.dino_chains_destroy(ctx, pool)
        dino.dino_unload_surrogate(ctx, sid)
    s1 = out["two_stage"]["stage1_acceptance"]
    out["two_stage"]["stage2_acceptance_given_stage1"] = (
        out["two_stage"]["acceptance"] / s1 if s1 else None)
    ctx.close()
    return out


def run_paper_shape(args, device=0):
    """The paper's network (6 x 400 GELU, r = 200 DIS, d_y = 25, N = 1681):
    proposals/s with the perturbation map (Cholesky of I + K K^T) and with the
    paper's eigen map (per-chain Jacobi eigendecomposition)."""
    import torch
    import dataclasses
    import paper_2403_08220_gb300 as dino
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device=device)
    ctx = dino.dino_init(device, 0, stream.cuda_stream, 0)
    out = {}
    for name, noise, C in (("paper_ndr_bf16", "perturbation", 16384),
                           ("paper_ndr_bf16", "eigen", 4096),
                           ("paper_hyper_bf16", "perturbation", 16384)):
        w = dataclasses.replace(CONFIGS[name], noise_map=noise)
        sid = load_surrogate(dino, ctx, w)
        info = dino.dino_surrogate_query(ctx, sid)
        pool = dino.dino_chains_create(ctx, sid, C, w.dt, SEED_CHAINS)
        dino.dino_chains_step(ctx, pool, 3, stats=False)
        k = max(2, min(args.steps, 10))
        secs, _ = timed_repeats(dino, ctx, pool, k, stream, lambda: None, 3)
        out[f"{name}/{noise}"] = {"chains": C, "proposals_per_s": C * k / secs,
                                  "ms_per_step": 1e3 * secs / k,
                                  "jacobian_mode": "forward" if info["jac_forward"] else "reverse",
                                  "d_y": w.d_y, "N": w.N}
        dino.dino_chains_destroy(ctx, pool)
        dino.dino_unload_surrogate(ctx, sid)
    ctx.close()
    return out


def serving_workload(n_surrogates=16, seed=2024):
    """Resident surrogates of the serving mix: r ~ U{32..400}, d_y ~ U{50..400}, r-2r-2r-d_y GELU."""
    from workloads import ACT_GELU, BASIS_DIS, Workload
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_surrogates):
        r = int(rng.integers(32, 401))
        dy = int(rng.integers(50, 401))
        out.append(Workload(f"serve_{k}", n_grid=65, r=r, widths=[r, 2 * r, 2 * r, dy],
                            activation=ACT_GELU, basis_kind=BASIS_DIS, n_chains=0, n_steps=0,
                            precision="bf16", seed_offset=1000 + 10 * k))
    return out


def run_serving(args, device=0):
    """Continuous batching under Poisson arrivals: p50/p99 latency and proposals/s.

    Latency is measured on the host: from the submit call to the poll that
    returns the request's outputs.  Two runs on the same resident surrogates:
    * stable load: chains log-uniform in [256, 8192] as written, steps uniform
      in [10, 100] (the written 1k-10k scaled down 100 times so that the run
      drains), arrivals at 0.7 of the capacity measured just before on a
      batch of such requests;
    * written load: 20 requests/s, chains log-uniform in [256, 8192], steps
      uniform in [1000, 10000], for a fixed window (60 s by default).  The
      offered work is far above one GPU's capacity, so the queue grows; the
      latencies of completed requests are reported with the ages of the ones
      still queued or running when the window closes (lower bounds of their
      latency), the queue length and the offered GPU-seconds per second.
    """
    import torch
    import paper_2403_08220_gb300 as dino
    torch.cuda.set_device(device)
    ws = serving_workload(args.serve_surrogates)
    rng = np.random.default_rng(7)

    def draw(lo_c, hi_c, lo_s, hi_s):
        k = int(rng.integers(0, len(ws)))
        C = int(np.exp(rng.uniform(np.log(lo_c), np.log(hi_c))))
        return k, C, int(rng.integers(lo_s, hi_s + 1))

    def run(ctx, sids, rate, window, lo_c, hi_c, lo_s, hi_s, max_requests, drain):
        outstanding, done = {}, []
        t_start = time.perf_counter()
        t_next = t_start
        n = 0
        while True:
            now = time.perf_counter()
            open_ = now - t_start <= window and n < max_requests
            if not open_ and (not drain or not outstanding):
                break
            if open_ and now >= t_next:
                k, C, S = draw(lo_c, hi_c, lo_s, hi_s)
                w = ws[k]
                t = dino.dino_serve_submit(ctx, sids[k], C, S, w.dt, 15 + n, w.r, w.N)
                outstanding[t] = (time.perf_counter(), C * S)
                n += 1
                t_next += rng.exponential(1.0 / rate)
            for t in list(outstanding):
                o = dino.dino_serve_poll(ctx, t)
                if o is not None:
                    t0, work = outstanding.pop(t)
                    done.append((time.perf_counter() - t0, work))
            time.sleep(0.001)
        return done, outstanding, time.perf_counter() - t_start, n

    def pct(x, q):
        return float(np.percentile(x, q)) if len(x) else None

    ctx = dino.dino_init(device, 0, None, 0)
    t0 = time.perf_counter()
    sids = [load_surrogate(dino, ctx, w) for w in ws]
    setup_s = time.perf_counter() - t0
    dino.dino_serve_config(ctx, n_streams=8, steps_per_round=4, max_active=32)
    # capacity on a batch of stable-size requests submitted at once
    cal, _, cal_s, _ = run(ctx, sids, 1e9, 1e9, 256, 8192, 10, 100, 24, True)
    capacity = sum(wk for _, wk in cal) / cal_s
    mean_work = float(np.mean([wk for _, wk in cal]))
    rate = 0.7 * capacity / mean_work
    st, _, st_s, _ = run(ctx, sids, rate, args.serve_window, 256, 8192, 10, 100, 10 ** 6, True)
    lat = np.array([l for l, _ in st])
    stable = {"offered_load_of_capacity": 0.7, "rate_per_s": rate, "requests": len(st),
              "p50_s": pct(lat, 50), "p99_s": pct(lat, 99),
              "proposals_per_s": sum(wk for _, wk in st) / st_s,
              "capacity_proposals_per_s": capacity,
              "request": "chains log-uniform [256, 8192], steps U[10, 100] (written 1k-10k / 100)"}
    ctx.close()

    ctx = dino.dino_init(device, 0, None, 0)
    sids = [load_surrogate(dino, ctx, w) for w in ws]
    dino.dino_serve_config(ctx, n_streams=8, steps_per_round=4, max_active=32)
    window = args.serve_written_window
    wr, left, wr_s, n = run(ctx, sids, 20.0, window, 256, 8192, 1000, 10000, 10 ** 6, False)
    t_end = time.perf_counter()
    status = dino.dino_serve_status(ctx)
    lat_w = np.array([l for l, _ in wr])
    ages = np.array([t_end - t0 for t0, _ in left.values()])
    works = [wk for _, wk in wr] + [wk for _, wk in left.values()]
    written = {"rate_per_s": 20.0, "window_s": window, "submitted": n,
               "completed": len(wr), "queued_at_end": status["queued"],
               "resident_at_end": status["active"], "peak_resident": status["peak_active"],
               "peak_hbm_gb": status["peak_hbm_used"] / 1e9,
               "p50_s": pct(lat_w, 50), "p99_s": pct(lat_w, 99),
               "completed_proposals_per_s": sum(wk for _, wk in wr) / wr_s,
               "unfinished_age_p50_s": pct(ages, 50), "unfinished_age_p99_s": pct(ages, 99),
               "unfinished_age_max_s": float(ages.max()) if len(ages) else None,
               "offered_gpu_s_per_s": float(20.0 * np.mean(works) / capacity) if works else 0.0,
               "request": "chains log-uniform [256, 8192], steps U[1000, 10000]",
               "note": "latencies of completed requests; unfinished requests' ages are lower "
                       "bounds of their latencies (censored at the window's end)"}
    t_close = time.perf_counter()
    ctx.close()   # cancels what is still queued; lets resident rounds finish
    written["close_s"] = time.perf_counter() - t_close
    return {"surrogates": len(ws), "r": [w.r for w in ws], "d_y": [w.d_y for w in ws],
            "setup_s": setup_s, "stable": stable, "written_load": written}


def cpu_baseline(args, sample_chains=None, sample_steps=None):
    """The FP64 oracle, untuned, on a bounded sample of the same workload."""
    from oracle import mlp, mmala, prior
    from oracle.chains import OracleChains
    w = CONFIGS[args.workload]
    inp = surrogate_inputs(w)
    if w.basis_kind == BASIS_KLE:
        E, D = prior.kle_basis(w.n_grid, w.prior_gamma, w.prior_delta, w.r)
    else:
        E, D = prior.dis_basis(w.n_grid, w.prior_gamma, w.prior_delta, inp["G"])
    f0, _ = mlp.forward(inp["Ws"], inp["bs"], w.activation, inp["m_true_r"])
    y, nv = make_data(f0, inp["eps"], w.noise_frac)
    sur = mmala.Surrogate(Ws=inp["Ws"], bs=inp["bs"], act=w.activation, y=y, noise_var=nv)
    C = sample_chains or 64
    K = sample_steps or 2
    if w.noise_map not in ("cholesky", "perturbation"):
        raise ValueError(f"workload {w.name} must name its proposal noise map")
    och = OracleChains(sur, E, D, w.n_grid, w.prior_gamma, w.prior_delta, C, w.dt,
                       seed=SEED_CHAINS, noise=w.noise_map)
    t0 = time.perf_counter()
    och.step(K)
    el = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": C * K / el, "unit": "proposals/s", "cores": cores, "kind": "oracle",
            "sample": f"{C} chains x {K} steps of {args.workload} ({el:.1f} s)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="r200_dis_bf16")
    ap.add_argument("--chains", type=int, default=0)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-mixing", action="store_true")
    ap.add_argument("--repeats", type=int, default=5)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-chains", type=int, default=512)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-hetero", action="store_true",
                    help="skip the eight-posterior heterogeneous batch")
    ap.add_argument("--hetero-r", type=int, default=0,
                    help="step only the heterogeneous posterior with this r (profiling)")
    ap.add_argument("--no-da", action="store_true", help="skip the delayed-acceptance line")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-shaped network line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving load test")
    ap.add_argument("--serve-window", type=float, default=10.0)
    ap.add_argument("--serve-written-window", type=float, default=60.0)
    ap.add_argument("--serve-surrogates", type=int, default=16)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank != 0:
            return
        w = CONFIGS[args.workload]
        per_step = []
        for _ in range(args.warmup):
            cpu_baseline(args, 8, 1)
        for _ in range(args.steps):
            per_step.append(cpu_baseline(args, 8, 1))
        v = statistics.median([p["value"] for p in per_step])
        cb = dict(per_step[0])
        cb["value"] = v
        cb["sample"] = f"8 chains x 1 step of {args.workload} per timed step"
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "proposals/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * 8 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: FP64 oracle on host cores",
                       "chains_per_step": 8, "r": w.r},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "proposals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return

    line = run_ours(args, rank, world, local)
    if rank == 0 and not args.no_hetero and world == 1:
        line["hetero"] = run_hetero(args, local)
    if rank == 0 and not args.no_da and world == 1:
        line["delayed_acceptance"] = run_da(args, local)
    if rank == 0 and not args.no_paper and world == 1:
        line["paper_shape"] = run_paper_shape(args, local)
    if rank == 0 and not args.no_serve and world == 1:
        line["serving"] = run_serving(args, local)
    if rank == 0:
        if not args.skip_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(args, args.cpu_chains, args.cpu_steps)
        print(json.dumps(line))


if __name__ == "__main__":
    main()
