#!/usr/bin/env python
"""Benchmark of the DDA hot path on one GB300 (or N replicas under torchrun).

Workload: sphere x = 40, m = 1.05 (LDR polarizability) on a 134^3 box
(1,260,552 dipoles, about 10 dipoles per wavelength, the paper's rule of
Sec. 3.1), padded FFT grid 270^3, incidence along z with x polarisation.

One step = one whole pass of the path for that particle: beta and the
right-hand side, the D-matrix (FFT of G in double-float, FP64-class, plus its
complex64 copy), QMR-CS in the FP32-refined form to a true relative residual
of 1e-5 (complex64 inner solve, double-float residual product), and the
scattering quantities (F at 181 angles in the xz plane, Q_ext, Q_abs).

value = products with A (complex64 and double-float) per second over the
timed steps, whole job.  Beside it: the time to residual 1e-5 of the same solve and
of the plain FP64 form on the same GPU, per-kernel roofline data, the CPU
oracle baseline and an end-to-end run through the C-ABI with host buffers.

--impl reference times the CPU oracle (the plain complex128 restatement of
the method) on bounded samples of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DDA matvecs/s & time-to-residual-1e-5 vs plain FP64 form on same GB300"
UNIT = "matvec/s"
N_SPHERE, X_SIZE, M_INDEX = 134, 40.0, 1.05
TOL = 1e-5
# inner complex64 solves stop at 8e-6 of the current residual: above the
# complex64 rounding floor of this problem (5e-6 to 7.5e-6 measured), so one
# FP64-class refinement step normally ends the solve below TOL
INNER_TOL = 8e-6
N_ANGLES = 181


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--steps-only", action="store_true",
                    help="run only the warm-up and timed steps (for profilers)")
    ap.add_argument("--inner-tol", type=float, default=INNER_TOL)
    ap.add_argument("--n", type=int, default=N_SPHERE, help=argparse.SUPPRESS)
    ap.add_argument("--workload", default="sphere134",
                    choices=["sphere134", "batch128", "sphere", "baselines", "products", "precond"],
                    help="sphere134: the headline line; batch128: the seeded 128-particle "
                         "batch (16 right-hand sides each), all right-hand sides to 1e-5; "
                         "sphere: one sphere (--n, --x, --m) solved once in each form; "
                         "baselines (with --impl reference): the CPU oracle's timings; "
                         "products: --products products of one precision (--prec) on the "
                         "sphere (--n, --x, --m), for profilers")
    ap.add_argument("--train-count", type=int, default=128,
                    help="precond workload: training particles (64^3 boxes)")
    ap.add_argument("--pc-maxiter", type=int, default=1500,
                    help="precond workload: Bi-CGSTAB iterations of each evaluation solve")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64", "df"],
                    help="products workload: complex64, complex128 or double-float product")
    ap.add_argument("--products", type=int, default=3, help="products workload: count")
    ap.add_argument("--box", default="",
                    help="products workload: an ellipsoid inscribed in an nx,ny,nz box instead of "
                         "the sphere (e.g. 100,100,540)")
    ap.add_argument("--engine", default="auto", choices=["auto", "stockham"],
                    help="products workload: FFT engine (register-resident passes where compiled, "
                         "or the shared-memory Stockham passes for every length)")
    ap.add_argument("--x", type=float, default=X_SIZE, help="sphere workload: size parameter")
    ap.add_argument("--m", type=float, default=M_INDEX, help="sphere workload: refractive index")
    ap.add_argument("--maxiter", type=int, default=100000, help="sphere workload: iteration cap")
    ap.add_argument("--forms", default="fp32_refined,fp64",
                    help="sphere workload: the forms to run (comma separated)")
    ap.add_argument("--inner-cap", type=int, default=0,
                    help="sphere workload: complex64 steps per inner solve before the switch to "
                         "complex128 vectors (0: the library's default)")
    ap.add_argument("--batch-count", type=int, default=128, help=argparse.SUPPRESS)
    ap.add_argument("--batch-threads", type=int, default=16,
                    help="host threads (particles in flight) of the batch workload")
    ap.add_argument("--batch-maxiter", type=int, default=20000)
    ap.add_argument("--batch-c64-only", type=int, default=0,
                    help="batch workload: 1 keeps the inner solves complex64 for the whole budget "
                         "(0, the default: the library's default switch after 1000 steps)")
    return ap.parse_args()


def workload_config(n, note):
    return {"workload": f"sphere x={X_SIZE:g} m={M_INDEX:g} LDR, {n}^3 box, QMR-CS to 1e-5 "
                        "(FP32-refined), F at 181 xz-plane angles",
            "n_box": n, "x": X_SIZE, "m": M_INDEX, "polarizability": "LDR",
            "solver": "qmr_cs", "precision": "fp32_refined", "tol": TOL,
            "l2": note, "parallelism": "replicas"}


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        # gpu_id: the UUID ("GPU-...") of the device in use; nvidia-smi does
        # not follow CUDA_VISIBLE_DEVICES, so an index could name another GPU
        self.idx = gpu_id
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "gpu": self.idx}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def load_mie(x, m):
    """Mie Q_ext and S11 at 0..180 degrees for a sphere of the workloads from
    tests/golden/mie_spheres.json (written by tests/golden/make_mie_golden.py
    from the oracle's Mie code); None for a sphere not in the file."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "mie_spheres.json")) as f:
            doc = json.load(f)
    except Exception:
        return None
    for c in doc["spheres"]:
        if abs(c["x"] - x) < 1e-12 and abs(c["m"] - m) < 1e-12:
            return {"qext": c["qext"], "theta_deg": doc["theta_deg"], "s11": np.asarray(c["s11"])}
    return None


def mie_errors(mie, qext, s11):
    """Sec. 3.1's error measures: relative Q_ext error, maximum and RMS (uniform
    over the 181 angles, both ends included) relative S11 error."""
    if mie is None:
        return None
    rel = np.abs(np.asarray(s11) - mie["s11"]) / mie["s11"]
    return {"qext_mie": mie["qext"], "qext_rel_err": abs(qext - mie["qext"]) / mie["qext"],
            "s11_max_rel_err": float(rel.max()), "s11_rms_rel_err": float(np.sqrt(np.mean(rel ** 2)))}


def working_launches(name, traced, c64_products, df_products):
    """Launches of a traced kernel that did work.  In the batched solver the
    right-hand side runs in blocks of 8 steps; the steps after convergence
    launch the complex64 product passes and QMR sweeps with every block
    returning at once (device skip mask), so those kernels are averaged over
    the products actually made; the double-float passes over the FP64-class
    products; everything else over its traced launches."""
    if name.endswith("_c64") or name.startswith("qmr_"):
        return min(traced, c64_products) if c64_products > 0 else traced
    if name.endswith("_df"):
        return min(traced, df_products) if df_products > 0 else traced
    return traced


def gpu_uuid(device_index):
    """nvidia-smi's id of a torch device: its UUID as 'GPU-<uuid>'."""
    import torch
    u = str(torch.cuda.get_device_properties(device_index).uuid)
    return u if u.startswith("GPU-") else "GPU-" + u


# ---------------------------------------------------------------- roofline models
def kernel_models(n, M, n_occ):
    """Algorithmic bytes (complex64 kernels, HBM-bound) and flops (complex128
    kernels, FP64-ALU-bound) per launch of each traced kernel, from the pass
    structure of the product (Sec. 2): padded M, lattice n, N_occ dipoles.
    FFT flops use 5 L log2 L per complex transform of length L."""
    lg = math.log2(M)
    out = {}
    for s, suf in ((8, "c64"), (16, "c128"), (16, "df")):
        bound = "hbm" if suf == "c64" else "alu"
        b1 = 3 * M * n * n * s          # [3][nz][ny][Mx]
        b2 = 3 * M * M * n * s          # [3][nz][My][Mx]
        oct_ = 6 * (M // 2 + 1) ** 3 * s
        vec = 3 * n_occ * s
        idx = n_occ * 3 + (n * n + 1) * 8   # x index (2 B) + material (1 B) per dipole + row offsets
        out[f"p1_xfft_{suf}"] = dict(bytes=vec + idx + b1, flops=3 * n * n * 5 * M * lg, bound=bound)
        out[f"p2_yfft_{suf}"] = dict(bytes=b1 + b2, flops=3 * n * M * 5 * M * lg, bound=bound)
        out[f"p3_zconv_{suf}"] = dict(bytes=2 * b2 + oct_, flops=3 * M * M * 2 * 5 * M * lg + 66 * M ** 3,
                                      bound=bound)
        out[f"p4_yifft_{suf}"] = dict(bytes=b2 + b1, flops=3 * n * M * 5 * M * lg, bound=bound)
        out[f"p5_xifft_{suf}"] = dict(bytes=b1 + 2 * vec + idx, flops=3 * n * n * 5 * M * lg,
                                      bound=bound)
    # QMR vector sweeps (complex64 inner solves): vt = pt - beta v (3 streams);
    # d, s, x, r updates and the next v, p (13 streams)
    vec8 = 3 * n_occ * 8
    out["qmr_k1"] = dict(bytes=3 * vec8, flops=0, bound="hbm")
    out["qmr_k2"] = dict(bytes=13 * vec8, flops=0, bound="hbm")
    # D build, register-resident passes with parity mirroring: x lines for
    # y, z <= M/2, y lines for kx, z <= M/2, z lines for kx, ky <= M/2;
    # all three passes per component
    h = M // 2 + 1
    lines = 3 * h * h
    out["dbuild_lines"] = dict(bytes=2 * lines * M * 16, flops=lines * 5 * M * lg, bound="alu")
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "of fallback"


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# stored ncu capture of the kernel as it is now (not measured by this run),
# with the capture it comes from.  Only valid for the 134^3 sphere on the
# 270^3 grid; None elsewhere, and removed whenever the kernel changes.
NCU_TRAFFIC_134 = {
    "p3_zconv_c64": (355240704 + 183284224,
                     "ncu --set full --clock-control none -k regex:fk_zconv -s 1 -c 1 of "
                     "python bench.py --workload products --n 134 --prec fp32 --products 3 "
                     "(fk_zconv<float, 15, 18, 16>, stored capture, not measured by this run)"),
}

FP64_PEAK_TFLOPS = 1.25   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe's nominal 1.25 TFLOP/s)


# ---------------------------------------------------------------- ranks
def reduce_over_ranks(t, counts, device):
    """Whole-job figures of one timed region over the ranks of the default
    process group: the slowest rank's time t and the sum of each count.
    Without a group of more than one rank, the values unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() < 2:
        return t, list(counts)
    tt = torch.tensor([float(t)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cc = torch.tensor([float(c) for c in counts], device=device, dtype=torch.float64)
    dist.all_reduce(cc, op=dist.ReduceOp.SUM)
    return float(tt.item()), [int(round(v)) for v in cc.tolist()]


def deal(items, rank, world):
    """The items rank `rank` of `world` works on: every world-th one, so the
    ranks share the work with no exchange (independent particles)."""
    return items[rank::world]


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_0704_0037_gb300 import build, dda, inputs

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n = args.n
    occ = inputs.sphere(n)
    prop = np.array([[0.0, 0.0, 1.0]])
    pol = np.array([[1.0, 0.0, 0.0]])
    th = inputs.angles_deg(N_ANGLES)
    t = np.deg2rad(th)
    dirs = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)], axis=1)
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR, prec=dda.DDA_FP32_REFINED, tol=TOL,
                maxiter=10000, inner_tol=args.inner_tol)
    p = dda.Particle(occ, [M_INDEX], X_SIZE, volume_corrected=True)
    P = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream()

    solve_ms = []

    def step(record=False):
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info, _ = dda.dda_solve(p.h, opts, prop, pol, P)
        e1.record(stream)
        F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P, prop, pol, dirs)
        if record:
            e1.synchronize()
            solve_ms.append(e0.elapsed_time(e1))
        return st, info[0], q

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(gpu_uuid(local_rank))
    if rank == 0:
        clocks.start()
    dda.dda_trace(p.h, True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    mv = mv64 = iters = 0
    last = None
    for _ in range(args.steps):
        st, info, q = step(record=True)
        mv += info["matvecs"]
        mv64 += info["matvecs_fp64"]
        iters += info["iters"]
        last = (st, info, q)
    # products that did work in the timed steps: complex64 (inner iterations)
    # and FP64-class (double-float residual products)
    c64_products, df_products = iters, mv64
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    trace = dda.dda_trace_read(p.h)
    dda.dda_trace(p.h, False)
    clk = clocks.stop() if rank == 0 else None
    t_max, (mv_all,) = reduce_over_ranks(ms, [mv], dev)
    value = mv_all / (t_max / 1e3)

    if args.steps_only:     # warm-up and timed steps only (for launch-list profiling)
        p.close()
        return {"metric": METRIC, "value": value, "unit": UNIT, "steps_only": True,
                "gpu_launches": int(trace.get("all_launches", (0, 0))[1])} if rank == 0 else None

    # accuracy of the last timed step's solution, outside the timed region:
    # the native FP64 residual of P (the refined form's own exit residual
    # comes from the double-float product) and the errors against Mie
    mie = load_mie(X_SIZE, M_INDEX) if n == N_SPHERE else None
    res32_fp64 = float(dda.dda_residual(p.h, dda.DDA_LDR, P, prop, pol)[0])
    M32, _, _ = dda.dda_mueller_plane_sym(p.h, dda.DDA_LDR, P, th)
    acc32 = mie_errors(mie, float(last[2][0, 0]), M32[:, 0, 0])

    # plain FP64 form on the same GPU (the comparison base of the metric),
    # median of three solves
    opts64 = dict(opts, prec=dda.DDA_FP64)
    fp64_runs = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64, info64, _ = dda.dda_solve(p.h, opts64, prop, pol, P)
        e1.record(stream)
        e1.synchronize()
        fp64_runs.append(e0.elapsed_time(e1))
    fp64_ms = statistics.median(fp64_runs)
    F64, q64 = dda.dda_scatter(p.h, dda.DDA_LDR, P, prop, pol, dirs[:1])
    res64_fp64 = float(dda.dda_residual(p.h, dda.DDA_LDR, P, prop, pol)[0])
    M64, _, _ = dda.dda_mueller_plane_sym(p.h, dda.DDA_LDR, P, th)
    acc64 = mie_errors(mie, float(q64[0, 0]), M64[:, 0, 0])

    # matvec-only rates (CUDA events, 10 products each, inputs > L2)
    rates = {}
    for prec, dt, nm in ((dda.DDA_FP32_REFINED, torch.complex64, "c64"),
                         (dda.DDA_FP64, torch.complex128, "c128"),
                         (dda.DDA_FP64_PAIR, torch.complex128, "df")):
        x = torch.randn((1, 3, p.n_occ), dtype=dt, device=dev)
        y = torch.empty_like(x)
        dda.dda_matvec(p.h, prec, x, y)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        reps = 10 if nm != "c128" else 3
        a.record(stream)
        for _ in range(reps):
            dda.dda_matvec(p.h, prec, x, y)
        b.record(stream)
        b.synchronize()
        rates[nm] = reps / (a.elapsed_time(b) / 1e3)
        del x, y

    result = None
    if rank == 0:
        st, info, q = last
        M = p.grid[0]
        models = kernel_models(n, M, p.n_occ)
        peaks, peak_note = load_peaks()
        ker = {k: v for k, v in trace.items() if k != "all_launches"}
        tot = sum(v[0] for v in ker.values())
        dom = max(ker, key=lambda k: ker[k][0])
        dms, dtraced = ker[dom]
        dcnt = working_launches(dom, dtraced, c64_products, df_products)
        avg_s = dms / dcnt / 1e3
        md = models.get(dom)
        if md and md.get("bound") == "hbm":
            achieved = md["bytes"] / avg_s / 1e9
            tr = NCU_TRAFFIC_134.get(dom) if n == N_SPHERE else None
            roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": tr[0] if tr else None,
                    "traffic_source": tr[1] if tr else "no stored capture of the current kernel",
                    "algorithmic_bytes": md["bytes"], "peak_note": f"hbm_gbs {peak_note}"}
        else:
            achieved = md["flops"] / avg_s / 1e12 if md else None
            roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                    "traffic": None, "peak_note": "FP64 ALU peak derived from unit counts and clock"}
        roof["share"] = dms / tot
        roof["avg_launch_ms"] = dms / dcnt
        roof["launches_traced"] = dtraced
        roof["launches_working"] = dcnt
        per_kernel = {}
        for k, (kms, kt) in sorted(ker.items(), key=lambda kv: -kv[1][0]):
            kc = working_launches(k, kt, c64_products, df_products)
            e = {"ms": round(kms, 3), "launches": kt, "working_launches": kc,
                 "share": round(kms / tot, 4), "avg_ms": round(kms / kc, 4)}
            md = models.get(k)
            if md and md.get("bound") == "hbm":
                e["hbm_gbs"] = round(md["bytes"] / (kms / kc / 1e3) / 1e9, 1)
                e["hbm_frac"] = round(e["hbm_gbs"] / peaks["hbm_gbs"], 3)
            elif md:
                e["fp64_class_tflops"] = round(md["flops"] / (kms / kc / 1e3) / 1e12, 3)
            per_kernel[k] = e
        c64_matvec_bytes = sum(models[f"p{i}_{nm}_c64"]["bytes"] for i, nm in
                               ((1, "xfft"), (2, "yfft"), (3, "zconv"), (4, "yifft"), (5, "xifft")))
        t2r = statistics.median(solve_ms) / 1e3
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+df+f64",
            "data": "synthetic (sphere occupancy computed from the lattice; no dataset)",
            "config": workload_config(n, "inputs larger than L2: 234 MB complex64 y-pass buffer, "
                                         "315 MB FP64 G grid, 121 MB D octant, per step"),
            "time_to_residual_s": t2r,
            "fp64_form": {"time_to_residual_s": fp64_ms / 1e3,
                          "runs_s": [round(v / 1e3, 5) for v in fp64_runs],
                          "status": info64[0]["status_name"],
                          "iters": info64[0]["iters"], "matvecs": info64[0]["matvecs"],
                          "rel_res_true": info64[0]["rel_res_true"],
                          "rel_res_fp64_check": res64_fp64, "qext": float(q64[0, 0]),
                          "vs_mie": acc64},
            "speedup_vs_fp64_form": (fp64_ms / 1e3) / t2r,
            "solve": {"status": info["status_name"], "iters_inner": info["iters"],
                      "outer": info["outer"], "matvecs": info["matvecs"],
                      "matvecs_fp64": info["matvecs_fp64"], "rel_res_true": info["rel_res_true"],
                      "rel_res_fp64_check": res32_fp64,
                      "qext": float(q[0, 0]), "qabs": float(q[0, 1]), "vs_mie": acc32,
                      "vs_fp64_form": {"qext_rel": abs(float(q[0, 0]) - float(q64[0, 0]))
                                       / abs(float(q64[0, 0])),
                                       "qabs_abs": abs(float(q[0, 1]) - float(q64[0, 1])),
                                       "s11_max_rel": float(np.max(np.abs(M32[:, 0, 0] - M64[:, 0, 0])
                                                                   / M64[:, 0, 0]))}},
            "matvec_only": {"c64_per_s": rates["c64"], "c128_per_s": rates["c128"],
                            "double_float_per_s": rates["df"],
                            "c64_effective_hbm_frac": c64_matvec_bytes * rates["c64"] / 1e9 / peaks["hbm_gbs"]},
            "roofline": roof,
            "kernels": per_kernel,
            "gpu_launches": int(trace.get("all_launches", (0, 0))[1]),
            "clocks": clk,
        }
    if not args.no_e2e:
        e2e = run_e2e(args, occ, opts, prop, pol, dirs, world, dev)
        if result is not None:
            result["e2e"] = e2e
    p.close()
    return result


def run_e2e(args, occ, opts, prop, pol, dirs, world, dev):
    """The same metric through the C-ABI from host memory: lattice upload,
    D-matrix, solve, P copied back to pinned host memory, scattering results
    on the host, handle freed -- all inside the timed region."""
    import torch
    from paper_0704_0037_gb300 import dda
    steps = max(2, args.steps // 2)
    P_host = None
    mv = 0
    h2d = d2h = 0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        p = dda.Particle(occ, [M_INDEX], X_SIZE, volume_corrected=True)
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        P = torch.empty((1, 3, p.n_occ), dtype=torch.complex128, device=dev)
        st, info, _ = dda.dda_solve(p.h, opts, prop, pol, P)
        if P_host is None:
            P_host = torch.empty(P.shape, dtype=P.dtype, pin_memory=True)
        P_host.copy_(P)
        F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P, prop, pol, dirs)
        torch.cuda.synchronize()
        mv += info[0]["matvecs"]
        h2d = occ.nbytes + 16 + 6 * 8 * 2
        d2h = P_host.numel() * 16 + F.size * 16 + q.size * 8
        p.close()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    dt, (mv,) = reduce_over_ranks(dt, [mv], dev)
    return {"value": mv / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": steps, "s_per_step": dt / steps}


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(n, n_products):
    """Oracle (CPU, complex128, full unsymmetrised D, scipy.fft) on the
    workload: D build once, then n_products FFT products.  Returns
    (products/s over the products, D build seconds, cores)."""
    from oracle import dda as odda
    from oracle.fft_matvec import _WORKERS
    from paper_0704_0037_gb300 import inputs
    occ = inputs.sphere(n)
    n_occ = int((occ > 0).sum())
    from oracle import lattice
    prob = odda.Problem(occ, [M_INDEX], lattice.kd_volume_corrected(X_SIZE, n_occ))
    t0 = time.perf_counter()
    prob.dmat()
    t_d = time.perf_counter() - t0
    beta = prob.beta("ldr", (0, 0, 1), (1, 0, 0))
    mv = prob.matvec(beta, "fft")
    x = inputs.random_vectors(3, 1, n_occ)[0]
    t0 = time.perf_counter()
    for _ in range(n_products):
        x = mv(x)
    t_p = time.perf_counter() - t0
    return n_products / t_p, t_d, _WORKERS


def cpu_baseline(n):
    rate, t_d, cores = oracle_sample(n, 2)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"2 FFT products of the CPU oracle (complex128, full unsymmetrised D, scipy.fft) "
                      f"on the {n}^3 sphere after one D build ({t_d:.1f} s, not in the rate)"}


def cpu_model():
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.lower()
                if key.startswith("model name"):
                    return line.split(":", 1)[1].strip()
                if key.startswith("cpu part"):
                    part = line.split(":", 1)[1].strip()
                    return f"{arm_parts.get(part, 'Arm')} (CPU part {part})"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference_baselines(args):
    """The CPU oracle's measured baseline: FFT products per second on spheres
    of n = 16, 64, 128 and 134 (median of 5 after one warm-up; D built before),
    and its time to a true residual of 1e-5 for the 16^3 sphere (x = 3, m = 1.5,
    both polarisations; dense LU and QMR-CS) and the 134^3 sphere (x = 40,
    m = 1.05, x-polarised; QMR-CS with the FFT product).  The 128^3 m = 2
    sphere (tens of thousands of iterations) and the 536^3 sphere (host
    memory) are products only."""
    from oracle import dda as odda
    from oracle import lattice, solvers, system
    from oracle.fft_matvec import _WORKERS
    from paper_0704_0037_gb300 import inputs
    out = {"cores": _WORKERS, "cpu": cpu_model(), "products": {}, "time_to_1e-5": {}}
    for n, xs, m in ((16, 3.0, 1.5), (64, 10.0, 1.5), (128, 20.0, 2.0), (134, 40.0, 1.05)):
        occ = inputs.sphere(n)
        prob = odda.Problem(occ, [m], lattice.kd_volume_corrected(xs, int((occ > 0).sum())))
        t0 = time.perf_counter()
        prob.dmat()
        t_d = time.perf_counter() - t0
        beta = prob.beta("ldr", (0, 0, 1), (1, 0, 0))
        mv = prob.matvec(beta, "fft")
        x = inputs.random_vectors(3, 1, prob.n_occ)[0]
        mv(x)
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            mv(x)
            ts.append(time.perf_counter() - t0)
        out["products"][str(n)] = {"n_occ": prob.n_occ, "grid": list(prob.grid),
                                   "products_per_s": 1.0 / statistics.median(ts),
                                   "d_build_s": t_d}
    # 16^3 sphere: dense LU and QMR-CS, both polarisations
    occ = inputs.sphere(16)
    prob = odda.Problem(occ, [1.5], lattice.kd_volume_corrected(3.0, int((occ > 0).sum())))
    for method in ("dense", "fft"):
        t0 = time.perf_counter()
        res = odda.simulate(prob, 3.0, "ldr", solver="qmr_cs", tol=TOL, method=method)
        out["time_to_1e-5"][f"sphere16_{'dense_lu' if method == 'dense' else 'qmr_cs'}"] = {
            "s": time.perf_counter() - t0, "rhs": 2,
            "iters": [i.get("iters") for i in res["info"]], "qext": [float(v) for v in res["qext"]]}
    # 134^3 sphere, x-polarised, QMR-CS
    occ = inputs.sphere(134)
    prob = odda.Problem(occ, [1.05], lattice.kd_volume_corrected(40.0, int((occ > 0).sum())))
    t0 = time.perf_counter()
    res = odda.simulate(prob, 40.0, "ldr", pols=((1, 0, 0),), solver="qmr_cs", tol=TOL)
    out["time_to_1e-5"]["sphere134_qmr_cs"] = {
        "s": time.perf_counter() - t0, "rhs": 1, "iters": res["info"][0].get("iters"),
        "qext": float(res["qext"][0]), "note": "includes the D build"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    if args.workload == "baselines":
        return run_reference_baselines(args)
    n = args.n
    from oracle import dda as odda
    from oracle import lattice
    from oracle.fft_matvec import _WORKERS
    from paper_0704_0037_gb300 import inputs
    occ = inputs.sphere(n)
    n_occ = int((occ > 0).sum())
    prob = odda.Problem(occ, [M_INDEX], lattice.kd_volume_corrected(X_SIZE, n_occ))
    prob.dmat()
    beta = prob.beta("ldr", (0, 0, 1), (1, 0, 0))
    mv = prob.matvec(beta, "fft")
    x = inputs.random_vectors(3, 1, n_occ)[0]
    for _ in range(args.warmup):
        mv(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = mv(x)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = (f"each step one FFT product of the CPU oracle (complex128, full unsymmetrised D, "
              f"scipy.fft, {_WORKERS} threads) on the {n}^3 sphere; D built once before warm-up")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(n, "CPU run"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _WORKERS, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- batch workload
def run_batch(args, rank, world, local_rank):
    """The seeded batch of particles (inputs.batch_instances): every particle's
    D-matrix built and its 16 right-hand sides (8 incidence directions x 2
    polarisations, CLDR) solved to a true residual of 1e-5 with the batched
    FP32-refined QMR-CS; particles run in args.batch_threads parallel host
    threads, each on its own stream, largest x m first.  Under torchrun the
    particles are dealt to the ranks (no exchange).  One step = the whole batch."""
    import torch
    from paper_0704_0037_gb300 import build, dda, inputs
    build.build()
    torch.cuda.set_device(local_rank)
    inst = inputs.batch_instances(args.batch_count)
    mine = deal(inst, rank, world)
    opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_CLDR, prec=dda.DDA_FP32_REFINED, tol=TOL,
                maxiter=args.batch_maxiter, inner_tol=INNER_TOL)
    # With the library's defaults a refinement step that needs more than 1000
    # complex64 steps continues with complex128 vectors and double-float
    # products (converges the hard right-hand sides at several times the cost
    # per step); --batch-c64-only 1 keeps the inner solves complex64 for the
    # whole budget of batch_maxiter steps (the inner_cap option).
    if args.batch_c64_only:
        opts["inner_cap"] = args.batch_maxiter
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mv = mv64 = rhs_ok = rhs_all = 0
    worst_res = 0.0
    # hardest first (x m, then size) so the long solves start early
    mine = sorted(mine, key=lambda it: (-it["x"] * it["m"], -int((it["occ"] > 0).sum())))
    parts, Ps = [], []
    for it in mine:
        s = torch.cuda.Stream()
        p = dda.Particle(it["occ"], [it["m"]], it["x"], volume_corrected=True, stream=s)
        parts.append(p)
        Ps.append(torch.zeros((16, 3, p.n_occ), dtype=torch.complex128, device="cuda"))
    torch.cuda.synchronize()
    st, sts, infos = dda.dda_solve_many([p.h for p in parts], opts, [it["prop"] for it in mine],
                                        [it["pol"] for it in mine], Ps, n_threads=args.batch_threads)
    for k, p in enumerate(parts):
        for i in infos[k]:
            mv += i["matvecs"]
            mv64 += i["matvecs_fp64"]
            rhs_all += 1
            rhs_ok += int(i["status"] == 0)
            worst_res = max(worst_res, i["rel_res_true"])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for p in parts:
        p.close()
    del Ps
    dt, (mv, rhs_ok, rhs_all) = reduce_over_ranks(dt, [mv, rhs_ok, rhs_all], "cuda")
    if rank != 0:
        return None
    return {"metric": "aggregate products/s, seeded 128-particle batch (16 RHS each) to 1e-5",
            "value": mv / dt, "unit": "matvec/s", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+df+f64", "data": "synthetic (seeded particles)",
            "config": {"workload": f"{args.batch_count} seeded particles (sphere/ellipsoid/cube, "
                                   "x~U[2,15], m~U[1.05,2], 16-64 dipoles across), CLDR, "
                                   "8 directions x 2 polarisations, batched FP32-refined QMR-CS "
                                   "to 1e-5", "threads": args.batch_threads,
                       "maxiter": args.batch_maxiter, "parallelism": "threads+streams",
                       "inner": "complex64 only" if args.batch_c64_only else
                                "complex64, then complex128 + double-float after 1000 steps"},
            "time_to_converge_all_s": dt, "rhs_converged": rhs_ok, "rhs_total": rhs_all,
            "worst_rel_res_true": worst_res, "matvecs_fp64": mv64}


def run_sphere(args):
    """One sphere (n^3 box, size parameter x, real index m, LDR, x-polarised
    incidence along z) solved once with QMR-CS to a true residual of 1e-5 in the
    FP32-refined form and in the plain FP64 form, each timed with CUDA events
    around the solve (D-matrix built before; an untimed solve of 16 steps
    first, so that one-time costs -- kernel loading, attribute setting -- stay
    out of the timed one).  For the long solves of the high-index spheres
    (Table 1: tens of thousands of iterations)."""
    import torch
    from paper_0704_0037_gb300 import build, dda, inputs
    build.build()
    occ = inputs.sphere(args.n)
    prop = np.array([[0.0, 0.0, 1.0]])
    pol = np.array([[1.0, 0.0, 0.0]])
    p = dda.Particle(occ, [args.m], args.x, volume_corrected=True)
    dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
    P = torch.zeros((1, 3, p.n_occ), dtype=torch.complex128, device="cuda")
    out = {}
    forms = [f for f in (("fp32_refined", dda.DDA_FP32_REFINED), ("fp64", dda.DDA_FP64))
             if f[0] in args.forms.split(",")]
    for name, prec in forms:
        opts = dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR, prec=prec, tol=TOL,
                    maxiter=args.maxiter, inner_tol=INNER_TOL, inner_cap=args.inner_cap)
        dda.dda_solve(p.h, dict(opts, maxiter=16), prop, pol, P)   # warm-up, untimed
        P.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        st, info, _ = dda.dda_solve(p.h, opts, prop, pol, P)
        e1.record()
        e1.synchronize()
        F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P, prop, pol, np.array([[0.0, 0.0, 1.0]]))
        i = info[0]
        th = inputs.angles_deg(N_ANGLES)
        Mm, _, _ = dda.dda_mueller_plane_sym(p.h, dda.DDA_LDR, P, th)
        out[name] = {"time_to_residual_s": e0.elapsed_time(e1) / 1e3, "status": i["status_name"],
                     "iters": i["iters"], "matvecs": i["matvecs"], "matvecs_fp64": i["matvecs_fp64"],
                     "outer": i["outer"], "rel_res_true": i["rel_res_true"],
                     "rel_res_fp64_check": float(dda.dda_residual(p.h, dda.DDA_LDR, P, prop, pol)[0]),
                     "qext": float(q[0, 0]), "qabs": float(q[0, 1]),
                     "vs_mie": mie_errors(load_mie(args.x, args.m), float(q[0, 0]), Mm[:, 0, 0])}
    p.close()
    r = (out["fp64"]["time_to_residual_s"] / out["fp32_refined"]["time_to_residual_s"]
         if "fp64" in out and "fp32_refined" in out else None)
    return {"metric": "time to true residual 1e-5, FP32-refined form vs plain FP64 form",
            "value": out[forms[0][0]]["time_to_residual_s"], "unit": "s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+df", "data": "synthetic (sphere occupancy)",
            "config": {"workload": f"sphere x={args.x:g} m={args.m:g} LDR, {args.n}^3 box, "
                                   "QMR-CS to 1e-5", "n_box": args.n, "x": args.x, "m": args.m,
                       "n_occ": int(p.n_occ), "grid": list(p.grid), "maxiter": args.maxiter,
                       "inner_cap": args.inner_cap},
            "forms": out, "speedup_vs_fp64_form": r}


def run_products(args):
    """args.products interaction-matrix products (Eq. (3)) of one precision
    on the sphere (n^3 box, x, m; LDR, incidence +z) applied to a seeded
    random vector, after the D-matrix build and one untimed product; prints
    the mean time per product (CUDA events).  A small, fixed launch sequence
    for ncu captures of the product kernels."""
    import torch
    from paper_0704_0037_gb300 import build, dda, inputs
    build.build()
    if args.box:
        nx, ny, nz = (int(v) for v in args.box.split(","))
        occ = inputs.ellipsoid(nx, ny, nz)
    else:
        occ = inputs.sphere(args.n)
    engine = dda.DDA_ENGINE_STOCKHAM if args.engine == "stockham" else None
    p = dda.Particle(occ, [args.m], args.x, volume_corrected=True, engine=engine)
    prec = {"fp32": dda.DDA_FP32_REFINED, "fp64": dda.DDA_FP64, "df": dda.DDA_FP64_PAIR}[args.prec]
    dda.dda_build_Dmatrix(p.h, dda.DDA_FP64 if prec == dda.DDA_FP64 else dda.DDA_FP32_REFINED)
    dda.dda_set_beta(p.h, dda.DDA_LDR, [(0.0, 0.0, 1.0)], [(1.0, 0.0, 0.0)])
    dt = torch.complex64 if prec == dda.DDA_FP32_REFINED else torch.complex128
    x = torch.from_numpy(inputs.random_vectors(1, 1, p.n_occ)).to("cuda", dt)
    y = torch.empty_like(x)
    dda.dda_matvec(p.h, prec, x, y)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.products):
        dda.dda_matvec(p.h, prec, x, y)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / max(1, args.products)
    # per-pass times of the same products (CUDA events inside the library)
    dda.dda_trace(p.h, True)
    for _ in range(args.products):
        dda.dda_matvec(p.h, prec, x, y)
    torch.cuda.synchronize()
    trace = {k: round(v[0] / max(1, v[1]), 4) for k, v in dda.dda_trace_read(p.h).items()
             if k != "all_launches"}
    dda.dda_trace(p.h, False)
    tiles = list(dda.dda_get_pass_tiles(p.h, prec))
    p.close()
    return {"workload": "products", "n_box": args.n, "box": args.box or None, "grid": list(p.grid),
            "pass_tiles": tiles,
            "prec": args.prec,
            "engine": args.engine,
            "products": args.products, "ms_per_product": ms, "ms_per_pass": trace}


def run_precond(args):
    """The learned right preconditioner on the 128^3 sphere (x = 20, m = 2,
    LDR, 1,099,136 dipoles): train the network on args.train_count particles
    (ellipsoids and sphere clusters at 64^3, m in [1.5, 2.0]), then solve the
    sphere with flexible Bi-CGSTAB with and without it (double-float products,
    complex128 vectors, args.pc_maxiter iterations at most), and with the
    FP32-refined QMR-CS for the same number of products; report iterations,
    products, time, true residual and the errors against Mie of each."""
    import torch
    from paper_0704_0037_gb300 import build, dda, inputs, learned
    build.build()
    net = dda.PcNet(seed=704037)
    tr = learned.train(net, count=args.train_count,
                       log=lambda m: print(m, file=sys.stderr, flush=True))
    occ = inputs.sphere(128)
    prop, pol = [(0.0, 0.0, 1.0)], [(1.0, 0.0, 0.0)]
    th = inputs.angles_deg(N_ANGLES)
    mie = load_mie(20.0, 2.0)
    out = {}
    with dda.Particle(occ, [2.0], 20.0, volume_corrected=True) as p:
        dda.dda_build_Dmatrix(p.h, dda.DDA_FP32_REFINED)
        P = torch.zeros((3, p.n_occ), dtype=torch.complex128, device="cuda")

        def report(name, info, secs):
            F, q = dda.dda_scatter(p.h, dda.DDA_LDR, P[None], prop, pol, np.zeros((0, 3)))
            Mm, _, _ = dda.dda_mueller_plane_sym(p.h, dda.DDA_LDR, P[None], th)
            out[name] = {"status": info["status_name"], "iters": info["iters"],
                         "products": info["matvecs"], "seconds": secs,
                         "rel_res_true": info["rel_res_true"],
                         "rel_res_fp64_check": float(dda.dda_residual(p.h, dda.DDA_LDR, P[None], prop, pol)[0]),
                         "network_dropped_at": info.get("outer", 0) if name == "learned" else None,
                         "qext": float(q[0, 0]), "vs_mie": mie_errors(mie, float(q[0, 0]), Mm[:, 0, 0])}

        for name, nn in (("plain_bicgstab", None), ("learned", net)):
            P.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, info, _ = dda.dda_solve_pc(p.h, nn, dict(pol=dda.DDA_LDR, tol=TOL, maxiter=args.pc_maxiter),
                                           prop, pol, P)
            torch.cuda.synchronize()
            report(name, info, time.perf_counter() - t0)
        # QMR-CS (FP32-refined, the library's default solver) for the same product budget
        P.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info, _ = dda.dda_solve(p.h, dict(solver=dda.DDA_QMR_CS, pol=dda.DDA_LDR,
                                              prec=dda.DDA_FP32_REFINED, tol=TOL,
                                              maxiter=2 * args.pc_maxiter, inner_tol=INNER_TOL),
                                    prop, pol, P[None])
        torch.cuda.synchronize()
        report("qmr_cs_fp32_refined", info[0], time.perf_counter() - t0)
    net.close()
    return {"metric": "learned right preconditioner: true residual and time, 128^3 sphere x=20 m=2",
            "unit": "s", "n_gpus": 1, "data": "synthetic (seeded particles and sphere)",
            "config": {"workload": "sphere x=20 m=2 LDR, 128^3 box (1,099,136 dipoles), tol 1e-5",
                       "pc_maxiter": args.pc_maxiter, "network_parameters": 1033430},
            "training": tr, "solves": out}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res))
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend="nccl")
    if args.workload == "products":
        print(json.dumps(run_products(args)))
        return
    if args.workload == "precond":
        print(json.dumps(run_precond(args)))
        return
    if args.workload == "sphere":
        if rank == 0:
            print(json.dumps(run_sphere(args)))
        return
    if args.workload == "batch128":
        res = run_batch(args, rank, world, local_rank)
        if rank == 0 and res is not None:
            print(json.dumps(res))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        if world == 1 and not args.no_cpu_baseline and not args.steps_only:
            res["cpu_baseline"] = cpu_baseline(args.n)
        print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
