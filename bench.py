#!/usr/bin/env python
"""Throughput of the stabilized multilevel B-spline fast EFIE matvec on GB300.

Workload (default "sphere20"): PEC sphere of 20 wavelength diameter (radius
10 m at lambda = 1 m), geodesic class-I mesh of frequency 200 (800,000
triangles, 1,200,000 RWG unknowns, ~0.055 lambda edges), cubic B-splines
(p = 3, s = 7), 0.1 lambda grid spacing, 3 grid levels, complex FP32 far field
with an FP64 near field, 64 right-hand sides per batch.  One step is one batched
fast matvec over the 64 vectors (charges, anterpolation, upward transfers,
stabilized FFT translations on every grid level, downward transfers,
interpolation, FP64 near field).  Inputs are seeded complex Gaussian current
vectors; the working set (tens of GB) is far larger than L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "sphere20": dict(freq=200, radius=10.0, k=2 * np.pi, p=3, delta=0.1, levels=3, nrhs=64, precision="mixed"),
    "sphere10": dict(freq=100, radius=5.0, k=2 * np.pi, p=3, delta=0.1, levels=3, nrhs=64, precision="mixed"),
    "mlf": dict(freq=200, radius=0.1, k=2 * np.pi, p=3, delta=0.0008, levels=5, nrhs=64, precision="mixed"),
    "sphere6": dict(freq=60, radius=3.0, k=2 * np.pi, p=3, delta=0.1, levels=3, nrhs=16, precision="mixed"),
    "sphere4": dict(freq=40, radius=2.0, k=2 * np.pi, p=3, delta=0.1, levels=2, nrhs=16, precision="mixed"),
    "c1": dict(freq=8, radius=0.5, k=2 * np.pi, p=3, delta=0.1, levels=2, nrhs=1, precision="fp64"),
}
METRIC = "fast-EFIE matvecs/s at N~1.2M (20-wavelength PEC sphere)"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Non-tensor peaks from the unit counts and clocks of this part: 128 FP32 lanes
# per SM, one FMA (2 flops) each per clock, at the maximum SM clock;
# FP64 at NVIDIA's nominal 1.25 TFLOP/s for GB300.  Tensor peaks come from the
# measured BF16 GEMM rate times the nominal TF32/BF16 ratio (1.1 / 2.25
# PFLOP/s dense).
FP32_LANES_PER_SM = 128
FP64_TFLOPS_NOMINAL = 1.25
TF32_PER_BF16 = 1.1 / 2.25
TF32_SPLIT_TERMS = 3      # a_hi b_hi + a_hi b_lo + a_lo b_hi per FP32-accurate product
DF_INSTR_PER_CMAC = 48     # FP32 instructions of one double-float complex multiply-add (near field)


def fp32_peak_tflops(sm_max_mhz):
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12, sms


# DRAM bytes per launch of the class's main kernel from a one-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of this bench command on the
# same workload, keyed by (workload, kernel class); an entry holds only while
# that kernel is unchanged.  near_A: the k_near_rows_df8 launch of the A part
# (all 64 right-hand sides); translation_mac_top_tc: one top-level
# k_mac_top_tc2<2> launch (one chunk pair).
NCU_DRAM_BYTES_PER_LAUNCH = {
    ("sphere20", "near_A"): 174.58e9 + 1.26e9,
    ("sphere20", "translation_mac_top_tc"): 25.08e9 + 18.84e9,
}


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self, device_index):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        rows = [[c.strip() for c in r] for r in rows if r and r[0].strip() == str(device_index)]
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        out["sm_mhz"] = float(np.median(sm)) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def build_mesh(w):
    import efie_inputs as E
    return E.icosphere(w["freq"], w["radius"])


def algorithmic(w, info, levels, nrhs):
    """Algorithmic flops / bytes per batched matvec (nrhs vectors) per kernel class.
    Translation MAC: 8 flops per complex MAC, pairs x n^3 per channel,
    4 channels per right-hand side (the interaction-list levels count their
    pairs only, also when the tensor-core form runs dense tiles over them).  Near field: 8 flops per stored entry per
    right-hand side, and 16 bytes per stored complex entry once per batch."""
    top = min(L["level"] for L in levels)
    mac_flops = sum(8.0 * L["n_far_pairs"] * L["nfft"] ** 3 * 4 * nrhs for L in levels if L["level"] != top)
    mac_top_flops = sum(8.0 * L["n_far_pairs"] * L["nfft"] ** 3 * 4 * nrhs for L in levels if L["level"] == top)
    near_A_flops = 8.0 * info["near_nnz_A"] * nrhs
    near_V_flops = 8.0 * info["near_nnz_V"] * nrhs
    near_A_bytes = 16.0 * info["near_nnz_A"]
    near_V_bytes = 16.0 * info["near_nnz_V"]
    return {"translation_mac": ("flops", mac_flops), "translation_mac_top": ("flops", mac_top_flops),
            "translation_mac_top_tc": ("flops", mac_top_flops), "translation_mac_tc": ("flops", mac_flops),
            "near_A": ("flops", near_A_flops),
            "near_V": ("flops", near_V_flops), "near_A_bytes": near_A_bytes, "near_V_bytes": near_V_bytes}


def grid_bytes(info, levels, nrhs, vb):
    """Algorithmic HBM bytes per batched matvec of the grid kernels: every
    setup product read once per batch, every grid and spectrum written once
    and read once.  vb = bytes per complex far-field
    value (8 for complex FP32), moments are real with vb/2 bytes.
      anterpolation: moments + leaf grids written + currents and charges read
      interpolation: moments + leaf grids read + FP64 outputs written
      forward_fft / inverse_fft: grids and spectra of every level, once each
      upward: child grids read, parent grids written
      downward: parent grids read, child grids read and written (accumulated)"""
    ch = 4 * nrhs
    by = {L["level"]: L for L in levels}
    top, leaf = min(by), max(by)
    grid = lambda L: L["n_boxes"] * L["sp"] ** 3 * ch * vb
    spec = lambda L: L["n_boxes"] * L["nfft"] ** 3 * ch * vb
    mom = (3 * info["moment_entries_rwg"] + info["moment_entries_tri"]) * (vb // 2)
    nb = info["n_unknowns"] + info["n_triangles"]
    out = {
        "anterpolation": mom + grid(by[leaf]) + nb * nrhs * vb,
        "interpolation": mom + grid(by[leaf]) + nb * nrhs * 16,
        "forward_fft": sum(grid(L) + spec(L) for L in levels),
        "inverse_fft": sum(grid(L) + spec(L) for L in levels),
        "upward": sum(grid(by[l]) + grid(by[l - 1]) for l in by if l > top),
        "downward": sum(grid(by[l - 1]) + 2 * grid(by[l]) for l in by if l > top),
    }
    return out


def job_rate(local_s, units_per_rank, world, dist, device):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units in local_s seconds: the slowest rank's time (MAX over
    ranks after a barrier) divides the units of all ranks.  Returns
    (units per second, max seconds)."""
    import torch
    t = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
    if dist:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_s = float(t.item())
    return units_per_rank * world / total_s, total_s


def run_ours(args, w, rank, world, local_rank):
    import torch
    import __graft_entry__ as g
    import paper_2606_13482_gb300 as G
    g.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    V, T = build_mesh(w)
    prec = G.EFIE_MIXED if w["precision"] == "mixed" else G.EFIE_FP64
    t0 = time.time()
    h = G.EFIE(V, T, w["k"], w["p"], w["delta"], w["levels"], precision=prec)
    t_setup = time.time() - t0
    info, levels = G.plan(V, T, w["k"], w["p"], w["delta"], w["levels"])
    hi = h.info()
    info["moment_entries_rwg"], info["moment_entries_tri"] = hi["moment_entries_rwg"], hi["moment_entries_tri"]
    N = h.N
    R = args.nrhs or w["nrhs"]
    gen = torch.Generator().manual_seed(1234 + rank)
    xh = torch.complex(torch.randn((R, N), generator=gen, dtype=torch.float64),
                       torch.randn((R, N), generator=gen, dtype=torch.float64)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    x = xh.cuda()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        h.matvec(x, y)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = h.launch_count()
    clocks = ClockSampler(os.path.join(args.clocks_dir, f"clocks_rank{rank}.csv"))
    with clocks:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            h.matvec(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
    n_launch = h.launch_count() - n_launch0
    ms = e0.elapsed_time(e1)
    value, total_s = job_rate(ms / 1000.0, R * args.steps, world, dist, "cuda")
    # kernel-class times: a second pass of the same steps with per-class CUDA
    # events; while it records, the library runs the near field and the far
    # field one after the other (they share the GPU on two streams in the
    # timed pass), so each class's time is its own
    h.profile(True)
    for _ in range(args.steps):
        h.matvec(x, y)
    torch.cuda.synchronize()
    h.profile(False)
    prof = h.profile_read()
    # end-to-end through the C ABI with pinned host buffers (efie_matvec_host: chunked H2D,
    # matvec and D2H, copies overlapping the products)
    e2e = None
    if not args.no_e2e:
        h.matvec_host(xh, yh)  # allocates the handle's staging buffers
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            h.matvec_host(xh, yh)
        torch.cuda.synchronize()
        e2e_rate, _ = job_rate(time.perf_counter() - t0, R * max(1, args.steps), world, dist, "cuda")
        e2e = {"value": e2e_rate, "unit": "matvecs/s",
               "h2d_bytes_per_step": int(xh.numel() * 16), "d2h_bytes_per_step": int(yh.numel() * 16)}
    # rooflines: the dominant kernel class and every class against its bound
    peaks, psrc = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_pk, n_sms = fp32_peak_tflops(sm_max)
    mixed = w["precision"] == "mixed"
    tc_top = "translation_mac_top_tc" in prof
    # the translation classes run inside seconds-long steps, under the power
    # cap: the sustained BF16 rate is their denominator (burst when absent)
    bf16_pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    bf16_kind = "sustained" if "bf16_tflops_sustained" in peaks else "burst"
    tf32_pk = bf16_pk * TF32_PER_BF16 / TF32_SPLIT_TERMS
    alg = algorithmic(w, info, levels, R)

    def flop_bound(name):
        """(bound, peak TFLOP/s, peak source) of a flop-counted kernel class."""
        if name in ("translation_mac_top_tc", "translation_mac_tc"):
            return ("tensor", tf32_pk, f"{psrc} BF16 {bf16_kind} {bf16_pk:.1f} TFLOP/s x 1.1/2.25 "
                    f"(TF32/BF16 nominal) / {TF32_SPLIT_TERMS} split terms (FP32-accurate products)")
        if mixed and name in ("near_A", "near_V"):
            # double-float near field: 48 FP32 instructions per complex MAC (8 algorithmic flops)
            return ("alu", fp32_pk / 2.0 * 8.0 / DF_INSTR_PER_CMAC,
                    f"{n_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz instruction issue / "
                    f"{DF_INSTR_PER_CMAC} FP32 instructions per double-float complex MAC x 8 flops")
        if mixed:
            return ("alu", fp32_pk, f"{n_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {sm_max:.0f} MHz")
        return ("alu", FP64_TFLOPS_NOMINAL, "NVIDIA nominal FP64 (non-tensor) rate of GB300")

    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms_total, dom_launches) = dom
    roof = None
    vb = 8 if mixed else 16
    gb = grid_bytes(info, levels, R, vb)
    if dom_name in alg and alg[dom_name][0] == "flops":
        bound, peak, src = flop_bound(dom_name)
        achieved = alg[dom_name][1] * args.steps / (dom_ms_total / 1000.0) / 1e12
        roof = {"kernel": dom_name, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": NCU_DRAM_BYTES_PER_LAUNCH.get((args.workload, dom_name)),
                "peak_source": src, "launches_per_step": dom_launches / max(1, args.steps)}
        if dom_name in ("near_A", "near_V"):
            nb = alg[dom_name + "_bytes"] * args.steps / (dom_ms_total / 1000.0) / 1e9
            roof.update(hbm_achieved_gbs=nb, hbm_frac=nb / peaks["hbm_gbs"], hbm_peak_source=psrc)
    elif dom_name in gb:
        achieved = gb[dom_name] * args.steps / (dom_ms_total / 1000.0) / 1e9
        roof = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": NCU_DRAM_BYTES_PER_LAUNCH.get((args.workload, dom_name)), "peak_source": psrc,
                "launches_per_step": dom_launches / max(1, args.steps)}
    if roof is not None:
        roof["timing"] = ("CUDA events around the kernel class on its launching stream, in a profiling pass of "
                          "the same steps after the timed one (near and far field serialized in that pass)")
    kernel_rooflines = {}
    for name, b in gb.items():
        if name in prof and prof[name][0] > 0:
            gbs = b * args.steps / (prof[name][0] / 1000.0) / 1e9
            kernel_rooflines[name] = {"bound": "hbm", "bytes_per_step": b, "achieved": gbs, "unit": "GB/s",
                                      "peak": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"]}
    for name in ("near_A", "near_V", "translation_mac", "translation_mac_top", "translation_mac_top_tc",
                 "translation_mac_tc"):
        if name in prof and prof[name][0] > 0:
            bound, pk, _ = flop_bound(name)
            fl = alg[name][1] * args.steps / (prof[name][0] / 1000.0) / 1e12
            kernel_rooflines[name] = {"bound": bound, "flops_per_step": alg[name][1], "achieved": fl,
                                      "unit": "TFLOP/s", "peak": pk, "frac": fl / pk}
    line = {
        "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s * 1000.0 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": (("c64 far (top-level translation on tensor cores: tcgen05 TF32 with a 3-term split of every FP32 "
                   "operand) / double-float near (two FP32 words, 48-bit significand) / c128 assembly, projectors, "
                   "Krylov") if tc_top else "c64 far / double-float near / c128 assembly, projectors, Krylov")
                 if mixed else "c128",
        "data": "synthetic (seeded geodesic sphere mesh, seeded complex Gaussian currents)",
        "config": {"workload": args.workload, "n_unknowns": N, "n_triangles": int(T.shape[0]),
                   "diameter_wavelengths": 2 * w["radius"] * w["k"] / (2 * np.pi), "p": w["p"],
                   "grid_spacing_wavelengths": w["delta"] * w["k"] / (2 * np.pi), "grid_levels": w["levels"],
                   "nrhs_per_step": R, "precision": w["precision"], "parallelism": f"replicas{world}",
                   "l2": "working set >> L2 (no flush)", "setup_s": t_setup, "setup_phases_s": h.setup_times(),
                   "levels": [{k: L[k] for k in ("level", "s", "sb", "shat", "nfft", "n_boxes", "n_far_pairs",
                                                  "n_offsets")} for L in levels],
                   "near_nnz_A": info["near_nnz_A"], "near_nnz_V": info["near_nnz_V"]},
        "clocks": clocks.summary(local_rank),
        "e2e": e2e, "gpu_launches": int(n_launch), "roofline": roof,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "kernel_rooflines": kernel_rooflines,
    }
    if rank == 0 and not args.no_solve:
        line["time_to_solve"] = time_to_solve(G, torch)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    h.close()
    if dist:
        dist.destroy_process_group()
    return line


def time_to_solve(G, torch):
    """Wall time to a 1e-6 FP64 true residual, mixed form vs the plain FP64
    form on the same GPU: 4-lambda PEC sphere (geodesic frequency 40, 48,000
    RWG), p = 3, 0.1 lambda grid, 2 grid levels, 8 plane waves (theta = 90 deg,
    phi = 0, 45, ..., 315 deg, theta-hat polarisation), GMRES(100), x0 = 0.
    (At 1.2M unknowns the plain FP64 solve would take hours on this GPU's FP64
    pipes, so the comparison runs on this smaller sphere.)"""
    import efie_inputs as E
    V, T = E.icosphere(40, 2.0)
    kh, pol = E.azimuth_planewaves(8)
    out = {"workload": "sphere4 (4-lambda PEC sphere, 48,000 RWG, 8 plane waves)", "tol": 1e-6}
    for name, prec in (("mixed", G.EFIE_MIXED), ("fp64", G.EFIE_FP64)):
        h = G.EFIE(V, T, 2 * np.pi, 3, 0.1, 2, precision=prec, gmres_restart=100, max_iters=3000)
        b = h.rhs_planewave(kh, pol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info, rc = h.solve(b, tol=1e-6)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "iterations": [i["iterations"] for i in info],
                     "true_rel_residual_max": max(i["true_rel_residual"] for i in info),
                     "converged": all(i["converged"] for i in info)}
        h.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


# ----------------------------------------------------------------- CPU oracle
# A problem the oracle finishes: the 1,080-unknown sphere of the smoke test
# (radius 0.3 wavelength, geodesic frequency 6, p = 3, 0.07-wavelength grid,
# 2 grid levels), with the oracle's own near field.
SMALL_ORACLE = dict(freq=6, radius=0.3, k=2 * np.pi, p=3, delta=0.07, levels=2)


class OracleSample:
    """One bounded sample of a single-vector matvec of the CPU oracle (FP64,
    NumPy/SciPy, one thread) on a workload it cannot run whole.  Every stage
    runs the oracle's own expressions (or calls its functions) on seeded
    samples of its units, and the sample's time is scaled by the workload's
    unit counts:
      anterpolation, interpolation   S RWGs + S triangles  -> N + N_t
      forward / inverse transforms   4 boxes per level     -> boxes
      kernel spectra (the oracle     4 box offsets         -> distinct offsets
        recomputes them per product)
      translation multiply-adds      64 box pairs          -> box pairs
      upward / downward transfers    4 children per level  -> boxes
      near field                     the oracle's sparse near product on the
                                     1,080-unknown sphere  -> stored entries
    step() returns (estimated seconds of one full matvec, seconds the sample
    took); the sample is (seconds taken) / (estimate) of one matvec."""

    def __init__(self, w, seed=0):
        import efie_inputs as E
        from oracle import fastmv as ofm
        from oracle.bspline import S_REMOVE, open_knots, projector, restriction_matrix
        from oracle.geometry import build_rwg
        from oracle.moments import pulse_moments, rwg_moments
        from oracle.tree import build_tree
        self.ofm = ofm
        rng = np.random.default_rng(seed)
        V, T = E.icosphere(w["freq"], w["radius"])
        m = build_rwg(V, T)
        tr = build_tree(m, w["k"], w["p"], w["delta"], w["levels"])
        self.m, self.tr = m, tr
        D, top, p = tr.D, tr.top, w["p"]
        LD = tr.levels[D]
        S = 200
        self.S = S
        ridx = rng.choice(m.N, S, replace=False)
        tidx = rng.choice(m.Nt, S, replace=False)
        self.mr = rwg_moments(m, tr, subset=ridx)
        self.mt = pulse_moments(m, tr, subset=tidx)
        boxes = np.unique(np.concatenate([tr.rwg_box[ridx], tr.tri_box[tidx]]))
        bmap = {b: i for i, b in enumerate(boxes)}
        self.rb = np.array([bmap[b] for b in tr.rwg_box[ridx]])
        self.tb = np.array([bmap[b] for b in tr.tri_box[tidx]])
        self.j = E.complex_gaussian(S, seed + 1)
        self.rho = E.complex_gaussian(S, seed + 2)
        self.q = np.zeros((len(boxes), 4, LD.sp, LD.sp, LD.sp), dtype=np.complex128)
        # an oracle operator whose translation helpers this sample calls
        self.op = ofm.BsplineEFIE.__new__(ofm.BsplineEFIE)
        self.op.kernel, self.op.k = None, w["k"]
        self.levels = []
        for ell in range(D, top - 1, -1):
            Lv = tr.levels[ell]
            B = len(Lv.boxes)
            P = projector(open_knots(0.0, float(Lv.sp - p), Lv.sp, p), p, S_REMOVE[p])[0]
            ns, n = Lv.shat, 2 * Lv.shat - 1
            # box pairs and distinct offsets (exact on the top level, from 64
            # sampled target boxes below it)
            ijk = Lv.ijk
            xs = np.arange(B) if (ell == top and B <= 4096) else rng.choice(B, min(B, 64), replace=False)
            offs = []
            for x in xs:
                dif = np.abs(ijk - ijk[x]).max(axis=1)
                pd = np.abs(ijk // 2 - ijk[x] // 2).max(axis=1)
                sel = (dif >= 2) & ((pd <= 1) | (ell == top))
                offs.append(ijk[x] - ijk[sel])
            offs = np.concatenate(offs) if offs else np.zeros((0, 3), int)
            pairs = len(offs) * B / len(xs)
            uo = np.unique(offs, axis=0) if len(offs) else offs
            lev = dict(ell=ell, B=B, P=P, ns=ns, n=n, L=Lv, pairs=pairs, n_offsets=len(uo),
                       off_sample=uo[rng.choice(len(uo), min(4, len(uo)), replace=False)] if len(uo) else uo,
                       qb=E.complex_gaussian((4, 4, Lv.sp, Lv.sp, Lv.sp), seed + 3),
                       Q=E.complex_gaussian((64, 4, n, n, n), seed + 4),
                       Kh=E.complex_gaussian((n, n, n), seed + 5),
                       Racc=np.zeros((8, 4, n, n, n), dtype=np.complex128))
            if ell > top:
                pa = tr.levels[ell - 1]
                r_ = int(round(pa.delta / Lv.delta))
                Up = open_knots(-pa.sb * r_, (pa.s - p + pa.sb) * r_, pa.sp, p)
                lev["CL"] = restriction_matrix(Up, open_knots(-Lv.sb, (Lv.s - p) + Lv.sb, Lv.sp, p), p)
                lev["qc"] = E.complex_gaussian((4, 4, Lv.sp, Lv.sp, Lv.sp), seed + 6)
                lev["rp"] = E.complex_gaussian((4, pa.sp, pa.sp, pa.sp), seed + 7)
            self.levels.append(lev)
        # near field: the oracle's own sparse products on a problem it builds whole
        sw = SMALL_ORACLE
        Vs, Ts = E.icosphere(sw["freq"], sw["radius"])
        self.small = ofm.BsplineEFIE(build_rwg(Vs, Ts), sw["k"], sw["p"], sw["delta"], sw["levels"])
        self.xs_small = E.complex_gaussian(self.small.mesh.N, seed + 8)
        rows_per_box = np.bincount(tr.rwg_box, minlength=len(LD.boxes))
        tris_per_box = np.bincount(tr.tri_box, minlength=len(LD.boxes))
        ijk = LD.ijk
        nbr_r = np.array([rows_per_box[np.abs(ijk - ijk[b]).max(axis=1) <= 1].sum() for b in range(len(ijk))])
        nbr_t = np.array([tris_per_box[np.abs(ijk - ijk[b]).max(axis=1) <= 1].sum() for b in range(len(ijk))])
        self.nnzA = float(np.sum(rows_per_box * nbr_r))
        self.nnzV = float(np.sum(tris_per_box * nbr_t))
        self.N, self.Nt = m.N, m.Nt

    def step(self):
        ofm = self.ofm
        est, t_all = {}, time.perf_counter()

        def timed(fn):
            t = time.perf_counter()
            fn()
            return time.perf_counter() - t

        q, rb, tb, mr, mt = self.q, self.rb, self.tb, self.mr, self.mt

        def ant():
            q[:] = 0
            np.add.at(q, (rb, slice(0, 3)), self.j[:, None, None, None, None] * mr)
            np.add.at(q, (tb, 3), self.rho[:, None, None, None] * mt)

        def itp():
            np.einsum("ndabc,ndabc->n", mr, q[rb, :3])
            np.einsum("tabc,tabc->t", mt, q[tb, 3])

        scale = (self.N + self.Nt) / (2 * self.S)
        est["anterpolation"] = timed(ant) * scale
        est["interpolation"] = timed(itp) * scale
        for lev in self.levels:
            P, ns, n, ell = lev["P"], lev["ns"], lev["n"], lev["ell"]

            def fwd():
                qt = ofm.mode3(P, P, P, lev["qb"])
                np.fft.fftn(np.pad(qt, [(0, 0), (0, 0)] + [(0, n - ns)] * 3), axes=(-3, -2, -1))

            def inv():
                r = np.fft.ifftn(lev["Q"][:4], axes=(-3, -2, -1))[..., :ns, :ns, :ns]
                ofm.mode3(P.T, P.T, P.T, r)

            est[f"transforms_L{ell}"] = (timed(fwd) + timed(inv)) * lev["B"] / 4

            def kernels():
                L = lev["L"]
                t = np.arange(-(ns - 1), ns)
                idx = np.mod(t, n)
                for o in lev["off_sample"]:
                    Dv = o[None, None, None, :] * L.h + np.stack(np.meshgrid(t, t, t, indexing="ij"), -1) * L.Delta
                    Kc = np.zeros((n, n, n), dtype=np.complex128)
                    Kc[np.ix_(idx, idx, idx)] = self.op._kernel_fn(Dv)
                    np.fft.fftn(Kc)

            if len(lev["off_sample"]):
                est[f"kernel_spectra_L{ell}"] = timed(kernels) * lev["n_offsets"] / len(lev["off_sample"])

            def mac():
                for i in range(64):
                    lev["Racc"][i % 8] += lev["Kh"][None] * lev["Q"][i]

            est[f"translation_L{ell}"] = timed(mac) * lev["pairs"] / 64
            if "CL" in lev:
                CL = lev["CL"]

                def transfers():
                    for b in range(4):
                        ofm.mode3(CL, CL, CL, lev["qc"][b])
                        ofm.mode3(CL.T, CL.T, CL.T, lev["rp"])

                est[f"transfers_L{ell}"] = timed(transfers) * lev["B"] / 4
        sm = self.small
        x = self.xs_small
        tA = timed(lambda: sm.A_near @ x)
        tV = timed(lambda: sm.mesh.sigma_apply(sm.V_near @ sm.mesh.sigmaT_apply(x)))
        est["near_A"] = tA / max(sm.A_near.nnz, 1) * self.nnzA
        est["near_V"] = tV / max(sm.V_near.nnz, 1) * self.nnzV
        return sum(est.values()), time.perf_counter() - t_all, est

    def small_matvec(self, reps=3):
        """Seconds per full oracle matvec (BsplineEFIE.matvec) of the 1,080-unknown sphere."""
        self.small.matvec(self.xs_small)
        t = time.perf_counter()
        for _ in range(reps):
            self.small.matvec(self.xs_small)
        return (time.perf_counter() - t) / reps


def _oracle_worker(workload, seed, warmup, steps, go, q):
    """One process on one host core: set-up and warm-up steps, then (when the
    parent says go) `steps` timed sample steps started together with the other
    workers, then the full oracle matvec of the small sphere."""
    try:
        s = OracleSample(WORKLOADS[workload], seed)
        for _ in range(warmup):
            s.step()
        q.put(("ready", seed, None))
        go.wait()
        res = [s.step() for _ in range(steps)]
        q.put(("stepped", seed, None))
        t_small = s.small_matvec()
        q.put(("result", seed, {"est": [r[0] for r in res], "took": [r[1] for r in res], "stages": res[-1][2],
                                "small_s": t_small}))
    except Exception as e:  # reported by the parent
        q.put(("error", seed, repr(e)))


def run_oracle_processes(workload, n_proc, warmup, steps, limit_s=1800):
    """Runs n_proc single-threaded oracle workers (spawned processes) in
    parallel.  Returns (results, wall seconds of the timed steps)."""
    import multiprocessing as mp
    import queue
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                            "CUDA_VISIBLE_DEVICES")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    procs = []
    try:
        go, q = ctx.Event(), ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(workload, i, warmup, steps, go, q), daemon=True)
                 for i in range(n_proc)]
        for p in procs:
            p.start()
        deadline = time.perf_counter() + limit_s

        def collect(kind):
            got = {}
            while len(got) < n_proc:
                try:
                    k, seed, val = q.get(timeout=2)
                except queue.Empty:
                    if time.perf_counter() > deadline or not all(p.is_alive() for p in procs):
                        raise RuntimeError(f"oracle workers stopped before '{kind}'")
                    continue
                if k == "error":
                    raise RuntimeError("oracle worker failed: " + val)
                if k == kind:
                    got[seed] = val
            return got

        collect("ready")
        t0 = time.perf_counter()
        go.set()
        collect("stepped")
        wall = time.perf_counter() - t0
        res = list(collect("result").values())
    finally:
        for p in procs:
            if p.is_alive():
                p.join(timeout=5)
            if p.is_alive():
                p.terminate()
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return res, wall


def _oracle_rates(res, wall):
    """Aggregate rate: the matvec fractions all workers completed in the
    timed steps over the wall time of those steps."""
    done = sum(t / e for r in res for e, t in zip(r["est"], r["took"]))
    return done / wall


def cpu_baseline(workload):
    """The oracle on the host cores beside the GPU number: one sample step per
    core, all cores at once and then one core alone, plus the full oracle
    matvec of the 1,080-unknown sphere on all cores and on one core."""
    ncores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res_all, wall_all = run_oracle_processes(workload, ncores, 0, 1)
    res_one, wall_one = run_oracle_processes(workload, 1, 0, 1)
    v_all = _oracle_rates(res_all, wall_all)
    v_one = _oracle_rates(res_one, wall_one)
    small_all = sum(1.0 / r["small_s"] for r in res_all)
    small_one = 1.0 / res_one[0]["small_s"]
    return {"value": v_all, "unit": "matvecs/s", "cores": ncores, "kind": "oracle",
            "sample": ("one sample step per core of the oracle's stages on seeded samples (200 RWGs + 200 "
                       "triangles, 4 boxes, 4 box offsets and 64 box pairs per level, the near field's sparse "
                       "product on the 1,080-unknown sphere), scaled by the workload's unit counts"),
            "one_core": {"value": v_one, "cores": 1},
            "stages_s_one_core": res_one[0]["stages"],
            "full_oracle_matvec_small_sphere": {"n_unknowns": 1080, "matvecs_per_s_all_cores": small_all,
                                                "matvecs_per_s_one_core": small_one},
            "wall_s": time.perf_counter() - t0, "cpu": _cpu_model()}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for l in out.splitlines():
            if l.startswith("Model name"):
                return l.split(":", 1)[1].strip() + f" ({os.cpu_count()} cores on host)"
    except Exception:
        pass
    return f"{os.cpu_count()} cores"


def reference_arm(args, w):
    """The CPU oracle as it stands, timed on all host cores: one single-threaded
    process per core, each running `warmup` untimed and then exactly `steps`
    timed sample steps of a single-vector oracle matvec of the workload.  A
    step's work is the fraction (seconds taken) / (estimated seconds of a full
    matvec) of one matvec; the value is the matvec fractions all processes
    completed over the wall time of the timed steps."""
    ncores = os.cpu_count() or 1
    res, wall = run_oracle_processes(args.workload, ncores, args.warmup, args.steps)
    v = _oracle_rates(res, wall)
    cb = {"value": v, "unit": "matvecs/s", "cores": ncores, "kind": "oracle",
          "sample": (f"{ncores} processes x {args.steps} sample steps of the oracle's stages on seeded samples, "
                     "scaled by the workload's unit counts"),
          "matvec_fraction_per_step": float(np.mean([t / e for r in res for e, t in zip(r["est"], r["took"])])),
          "cpu": _cpu_model()}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "matvecs/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": args.workload, "nrhs_per_step": 1},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def batch_meshes():
    """Ten PEC ellipsoids, semi-axes uniform in [0.5, 3] wavelengths (seed 3),
    each a scaled geodesic sphere (30 f^2 unknowns at frequency f).  The
    unknown counts span 5,000 - 60,000: frequencies 13 ... 44 in ten even
    steps, the finer meshes on the larger ellipsoids."""
    import efie_inputs as E
    rng = np.random.default_rng(3)
    axes = [rng.uniform(0.5, 3.0, size=3) for _ in range(10)]
    freqs = [int(round(13 + i * 31 / 9)) for i in range(10)]
    order = np.argsort([a.max() for a in axes])
    out = [None] * 10
    for rank, i in enumerate(order):
        out[i] = E.ellipsoid(freqs[rank], tuple(axes[i]))
    return out


def run_batch(args):
    """Batched form: every ellipsoid's product in one CUDA graph launch, one
    plane wave on nine of them and 360 monostatic plane waves (azimuth, 1 degree
    steps, theta-hat polarisation) on the largest; mixed precision, p = 3,
    a 0.1-wavelength grid (0.12-0.16 on the coarsest meshes, whose edges
    exceed 0.1 wavelength), autotuned chunk and kernels per mesh."""
    import torch
    import __graft_entry__ as g
    import paper_2606_13482_gb300 as G
    import efie_inputs as E
    g.build()
    k = 2 * np.pi
    meshes = batch_meshes()
    hs, deltas, t0 = [], [], time.time()
    for V, T in meshes:
        # the finest grid of 0.1, 0.12, ... wavelengths that a coarse mesh's
        # protrusion allows with one buffer spline
        for delta in (0.1, 0.12, 0.14, 0.16, 0.18, 0.2):
            try:
                info, _ = G.plan(V, T, k, 3, delta, 1)
                break
            except G.EfieError:
                continue
        levels = max(1, min(3, info["depth"] - 1))
        hs.append(G.EFIE(V, T, k, 3, delta, levels, precision=G.EFIE_MIXED))
        deltas.append(delta)
    t_setup = time.time() - t0
    big = int(np.argmax([h.N for h in hs]))
    xs = []
    for i, h in enumerate(hs):
        kh, pol = E.azimuth_planewaves(360 if i == big else 1, 1.0)
        xs.append(h.rhs_planewave(kh, pol))
    for i, h in enumerate(hs):
        h.autotune(min(8, xs[i].shape[0]))
    ys = [torch.empty_like(x) for x in xs]
    b = G.Batch(hs)
    for _ in range(args.warmup):
        b.matvec(xs, ys)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        b.matvec(xs, ys)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the same products launched one handle at a time, for comparison
    e0.record(stream)
    for _ in range(args.steps):
        for h, x, y in zip(hs, xs, ys):
            h.matvec(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / args.steps
    nv = sum(x.shape[0] for x in xs)
    b.close()
    for h in hs:
        h.close()
    return {"metric": "batched fast-EFIE matvecs/s (10 ellipsoids, 369 right-hand sides, one graph launch)",
            "value": nv / (ms / 1000.0), "unit": "matvecs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 far / c128 near", "data": "synthetic (seeded ellipsoids, plane waves)",
            "config": {"workload": "batch10", "rwg_unknowns": [int(1.5 * T.shape[0]) for _, T in meshes],
                       "grid_spacing_wavelengths": deltas, "nrhs": [int(x.shape[0]) for x in xs],
                       "setup_s": t_setup},
            "sequential_ms_per_step": ms_seq, "graph_speedup": ms_seq / ms}


def precond_family(seed, n):
    """Seeded family of PEC scatterers meshed at ~0.1 wavelength along their
    longest axis: ellipsoids with semi-axes uniform in [0.6, 1.2] wavelengths,
    and every third member an ellipsoid plus a thin closed plate (thickness two
    edge lengths) beside it, separated by a seeded gap.  (Sized so that plain
    GMRES reaches a 1e-6 true residual within its iteration budget.)"""
    import efie_inputs as E
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        axes = rng.uniform(0.6, 1.2, size=3)
        freq = int(np.ceil(1.205 * axes.max() / 0.1))
        V, T = E.ellipsoid(freq, tuple(axes))
        if i % 3 == 2:
            lx, ly = rng.uniform(0.6, 1.2, size=2)
            gap = rng.uniform(0.3, 0.6)
            box = E.thin_box((lx, ly, 0.2), (int(np.ceil(lx / 0.1)), int(np.ceil(ly / 0.1)), 2),
                             center=(0.0, 0.0, axes[2] + gap + 0.1))
            V, T = E.merge_meshes((V, T), box)
        out.append((V, T))
    return out


def run_precond(args):
    """Learned preconditioner (not in the paper): the network is trained on
    residual/error pairs harvested from the plain solver's own GMRES runs on
    four training scatterers; then each of two held-out scatterers is solved
    for four plane waves in one batched call, to a 1e-6 FP64 true residual,
    three ways on the same GPU:
      learned  - FGMRES(100) + network, mixed precision (complex FP32 far field)
      mixed    - plain GMRES(100), mixed precision
      fp64     - plain GMRES(100), the plain FP64 form (FP64 far and near field)
    and the learned form is compared with the plain FP64 form."""
    import tempfile
    import torch
    import __graft_entry__ as g
    import paper_2606_13482_gb300 as G
    g.build()
    k = 2 * np.pi

    def planewaves(n, seed):
        r = np.random.default_rng(seed)
        kh = r.standard_normal((n, 3))
        kh /= np.linalg.norm(kh, axis=1, keepdims=True)
        pol = np.cross(kh, r.standard_normal((n, 3)))
        return kh, pol / np.linalg.norm(pol, axis=1, keepdims=True)

    def handle(V, T, precision):
        info, _ = G.plan(V, T, k, 3, 0.1, 1)
        return G.EFIE(V, T, k, 3, 0.1, max(1, min(3, info["depth"] - 1)), precision=precision,
                      gmres_restart=100, max_iters=4000)

    path = os.path.join(tempfile.mkdtemp(), "net.bin")
    train, test = precond_family(4, 4), precond_family(40, 2)
    t0 = time.time()
    losses = []
    for i, (V, T) in enumerate(train):
        h = handle(V, T, G.EFIE_MIXED)
        if i:
            h.precond_load(path)
            h.precond_enable(False)
        b = h.rhs_planewave(*planewaves(3, i))
        R, Ee = h.precond_harvest(b, restart=8, n_cycles=6)
        losses.append(h.precond_train(R, Ee, epochs=20, lr=2e-3, seed=i))
        h.precond_save(path)
        h.close()
    t_train = time.time() - t0
    rows = []
    for i, (V, T) in enumerate(test):
        res = {}
        for name, prec in (("learned", G.EFIE_MIXED), ("mixed", G.EFIE_MIXED), ("fp64", G.EFIE_FP64)):
            h = handle(V, T, prec)
            res["rwg_unknowns"] = int(h.N)
            b = h.rhs_planewave(*planewaves(4, 100 + i))
            if name == "learned":
                h.precond_load(path)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info, _ = h.solve(b, tol=1e-6)
            torch.cuda.synchronize()
            res[name] = {"seconds": time.perf_counter() - t1, "iterations": [d["iterations"] for d in info],
                         "true_rel_residual_max": max(d["true_rel_residual"] for d in info),
                         "converged": all(bool(d["converged"]) for d in info),
                         "fallback": [d["precond_fallback"] for d in info]}
            h.close()
        res["speedup_learned_vs_fp64"] = res["fp64"]["seconds"] / res["learned"]["seconds"]
        res["speedup_learned_vs_mixed"] = res["mixed"]["seconds"] / res["learned"]["seconds"]
        rows.append(res)
    return {"metric": "time to a 1e-6 true residual: learned-preconditioned mixed-precision batched form vs the "
                      "plain FP64 GPU form (held-out scatterers, 4 plane waves per batched solve)",
            "train_rwg_unknowns": [int(1.5 * T.shape[0]) for _, T in train], "train_seconds": t_train,
            "train_loss_first_last": [[round(l[0], 4), round(l[-1], 4)] for l in losses], "held_out": rows,
            "gmres_restart": 100, "data": "synthetic (seeded ellipsoids and plate unions)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere20", choices=sorted(WORKLOADS) + ["batch10", "precond"])
    ap.add_argument("--nrhs", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="folder for the raw nvidia-smi clock samples of the timed region")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload in ("batch10", "precond"):
        if args.impl == "ours" and rank == 0:
            print(json.dumps(run_batch(args) if args.workload == "batch10" else run_precond(args)), flush=True)
        return
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        if rank != 0:
            return
        line = reference_arm(args, w)
    else:
        line = run_ours(args, w, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
