#!/usr/bin/env python
"""Benchmark of the boundary-integral matvec (step 2(a) of the hybrid solver, Sec. II.E).

Headline workload: the large scatterer -- geodesic sphere of radius 20 wavelengths,
1,161,620 triangles (1,742,430 RWG per current, 3,484,860 unknowns J + M), 9-level MLFMA
at 3 digits, FP32 complex, eight seeded complex-Gaussian right-hand sides in one product,
op_mode 0 (the C block of Eq. 42).  One step = one full product Y = C X of the 8 columns.

Secondary sections on the same line: the 20,480-triangle sphere (61,440 unknowns, one RHS),
the batched monostatic sweep on the cube with cylinder (64 plane waves per product), and the
serving stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle (plain dense
Galerkin rows, Eqs. 43-46) on the host cores on a bounded sample of rows of the same
matrix, times the same 8 columns.  Multi-GPU runs are independent replicas (one operator
per GPU, no data exchange): value = total unknowns*RHS over the max time across ranks.
"""
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

METRIC = "BI matvec unknowns*RHS/s at rel.err<=1e-3 vs FP64"
UNIT = "unknowns*RHS/s"
K0 = 2 * np.pi
HEADLINE = dict(name="sphere_r20_nu241", nrhs=8,
                desc="large scatterer: PEC-sphere surface r=20 lambda, 1161620 triangles, 3484860 unknowns (J+M), "
                     "9-level MLFMA 3 digits, FP32, 8 RHS per product")
SECONDARY = dict(name="sphere_r2_nu32", nrhs=1,
                 desc="coated-sphere outer surface r=2 lambda, 20480 triangles, 61440 unknowns (J+M), 5-level MLFMA "
                      "3 digits, FP32, 1 RHS")
WORKLOAD = HEADLINE["desc"]
GOLDEN_C5 = os.path.join(ROOT, "tests", "golden", "c5_rows.json")
# FP32 FMA peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (maximum SM clock)
ALU_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=8, help="oracle rows in the CPU-baseline sample")
    ap.add_argument("--secondary", type=int, default=1, help="run the 61,440-unknown one-RHS section (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=64, help="RHS of the batched monostatic-sweep section (0: skip)")
    ap.add_argument("--sweep", type=int, default=1, help="solve the 180-incidence sweep end to end (0: skip)")
    ap.add_argument("--serving", type=int, default=64, help="requests of the serving section (0: skip)")
    ap.add_argument("--serving-max-unknowns", type=int, default=50000)
    ap.add_argument("--serving-max-rhs", type=int, default=32)
    ap.add_argument("--serving-plain", type=int, default=1, help="time the plain one-at-a-time form too (0: skip)")
    ap.add_argument("--serving-unshared", type=int, default=1,
                    help="time the server with one operator per request too (0: skip)")
    ap.add_argument("--profile-one", choices=["headline", "secondary", "cube_cylinder"],
                    help="profiling aid: set up the named workload, run a few products, then bracket ONE "
                         "product with cudaProfilerStart/Stop (for ncu --profile-from-start off) and exit")
    ap.add_argument("--nrhs", type=int, default=0, help="with --profile-one: right-hand sides (0: the workload's)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving section (e.g. the full c4 stream: --serving 500 "
                         "--serving-max-unknowns 200000 --serving-plain 0) and print its JSON")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_mesh(name=HEADLINE["name"]):
    from paper_2210_04892_gb300.inputs import workload
    v, t, meta = workload(name)
    return v, t, meta


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------- algorithmic bytes
def stage_bytes(info, nrhs, csize=8):
    """Algorithmic bytes of each stage of one product (every array touched once)."""
    N, nun = info["n_rwg"], info["n_unknowns"]
    lf = info["leaf_level"]
    E = 2 * nrhs
    vec = nun * nrhs * csize
    b = {}
    b["gather"] = 2 * vec + 4 * N
    b["near"] = info["near_pairs"] * 2 * csize + 2 * vec          # (A, B) per pair, x read, y write
    Kl = info["K"][lf]
    pat = N * (Kl // 2) * 2 * csize                                  # one pattern array (one of each antipodal pair)
    far = lambda l: info["boxes"][l] * info["K"][l] * E * csize
    b["aggregate"] = pat + vec + far(lf)
    b["interpolate"] = sum(far(l + 1) + far(l) for l in range(2, lf))
    b["translate"] = sum(2 * far(l) + 343 * info["K"][l] * csize for l in range(2, lf + 1))
    b["anterpolate"] = sum(far(l) + 2 * far(l + 1) for l in range(2, lf))
    b["receive"] = 2 * pat + far(lf) + vec
    b["scatter"] = 3 * vec + 4 * N
    return b


def stage_flops(info, nrhs, p=10):
    """Algorithmic floating-point operations of each stage (a complex multiply-add counts 8,
    a real-by-complex one 4; Lagrange passes with p taps per dimension)."""
    N, nun = info["n_rwg"], info["n_unknowns"]
    lf = info["leaf_level"]
    R, E = nrhs, 2 * nrhs
    f = {"gather": 0, "scatter": 0}
    f["near"] = info["near_pairs"] * R * 32                        # 4 complex MACs per pair and RHS
    f["aggregate"] = N * info["K"][lf] * R * 32                     # J and M into two components
    f["receive"] = N * info["K"][lf] * R * 64                       # 8 complex MACs per (RWG, direction, RHS)
    nth = lambda l: info["L"][l] + 1
    nph = lambda l: 2 * (info["L"][l] + 1)

    def level_pass(l):  # parent level l, children at l + 1
        nc = info["boxes"][l + 1]
        return nc * E * (nth(l) * nph(l + 1) * p * 4 + info["K"][l] * p * 4 + info["K"][l] * 8)
    f["interpolate"] = sum(level_pass(l) for l in range(2, lf))
    f["anterpolate"] = f["interpolate"]
    f["translate"] = sum(info["interactions"][l] * info["K"][l] * E * 8 for l in range(2, lf + 1))
    return f


def stage_roofline(info, nrhs, stages, hbm_gbs):
    """Per stage: the bound (HBM bytes or FP32 flops, whichever takes longer at the peaks),
    the achieved rate and its fraction of that peak.  Where the product fuses the gather of x
    into the near stage and the scatter of y into the receive (the gather and scatter stages
    then time as empty), their bytes move to those stages and they are not reported apart."""
    sb, sf = stage_bytes(info, nrhs), stage_flops(info, nrhs)
    stages = dict(stages)
    vec = info["n_unknowns"] * nrhs * 8
    if "gather" in stages and stages["gather"] < 0.01 * max(stages.get("near", 0.0), 1e-9):
        stages.pop("gather")
        sb["near"] += sb["gather"]
    if "scatter" in stages and stages["scatter"] < 0.01 * max(stages.get("receive", 0.0), 1e-9):
        stages.pop("scatter")
        sb["receive"] += vec          # the receive also reads the near part of y and writes y
    out = {}
    for k, ms in stages.items():
        t_hbm = sb[k] / (hbm_gbs * 1e9)
        t_alu = sf.get(k, 0) / (ALU_FP32_TFLOPS * 1e12)
        if t_alu > t_hbm:
            out[k] = {"ms": ms, "bound": "alu", "achieved": sf[k] / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                      "peak": ALU_FP32_TFLOPS, "frac": t_alu / (ms * 1e-3), "bytes": sb[k], "flops": sf.get(k, 0)}
        else:
            out[k] = {"ms": ms, "bound": "hbm", "achieved": sb[k] / (ms * 1e-3) / 1e9, "unit": "GB/s",
                      "peak": hbm_gbs, "frac": t_hbm / (ms * 1e-3), "bytes": sb[k], "flops": sf.get(k, 0)}
    return out


def launches_per_step(info, nrhs=1, tuned=""):
    """Kernels of one product on this path: near (side stream; with several right-hand sides
    preceded by the gather of x into tree order), aggregation, one interpolation and one
    anterpolation per level pair, one translation per level, receive.  `tuned` is the handle's
    tuned-form report (bi_tuned_config): a level pass tuned to a two-pass form launches two
    kernels (the theta pass and the phi pass)."""
    lf = info["leaf_level"]
    gather = 1 if nrhs > 1 else 0
    if lf < 2:
        return 2 + gather
    E = " E %d:" % (2 * nrhs)
    two_pass = sum(1 for line in tuned.splitlines()
                   if E in line and line.startswith(("interpolate", "anterpolate")) and "two-pass" in line)
    return 1 + 1 + (lf - 2) + (lf - 1) + (lf - 2) + 1 + gather + two_pass


def measured_traffic(name="dram_matvec_sphere_r2_61440.md"):
    """Per-launch DRAM bytes of the kernels from a committed ncu summary
    (lines `traffic: <stage> <kernel> <bytes>`); {} when absent."""
    out = {}
    p = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(p):
            if line.startswith("traffic:"):
                _, stage, kernel, nbytes = line.split()
                out[stage] = (kernel, int(nbytes))
    except OSError:
        pass
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------------- CPU oracle
def oracle_rows_rate(v, t, rows, x=None, y=None):
    """Time the oracle computing the given rows of the C block times the columns of x
    ([nrhs][nun]); returns (rows/s, seconds, rel. error of y[:, rows] when y is given)."""
    import oracle
    t0 = time.perf_counter()
    Z = oracle.rows(v, t, K0, 0, rows)
    ref = (Z @ x.T).T if x is not None else None
    dt = time.perf_counter() - t0
    err = None
    if y is not None:
        err = float(np.linalg.norm(y[:, rows] - ref) / np.linalg.norm(ref))
    return len(rows) / dt, dt, err


def golden_error(y):
    """Relative error of the headline product y ([nrhs][nun]) on the stored oracle rows
    (tests/golden/c5_rows.json, written by the oracle alone); None when the file is absent."""
    try:
        g = json.load(open(GOLDEN_C5))
    except OSError:
        return None
    ref = np.array(g["y"], np.float64)
    ref = ref[..., 0] + 1j * ref[..., 1]
    rows = np.array(g["rows"])
    return float(np.linalg.norm(y[:, rows] - ref) / np.linalg.norm(ref))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, sample_rows
    v, t, meta = workload_mesh()
    R = HEADLINE["nrhs"]
    nun = oracle.num_unknowns(v, t, 0)
    x = complex_gaussian(nun, R, seed=meta["seed"])
    # rows per step: the whole run stays within a few minutes
    probe = sample_rows(nun, 2, seed=SEED_BASE + 21)
    rate, _, _ = oracle_rows_rate(v, t, probe, x)
    budget = 150.0
    per_step = max(1, int(budget * rate / max(1, args.steps + args.warmup)))
    per_step = min(per_step, 64)
    rng_rows = [sample_rows(nun, per_step, seed=SEED_BASE + 100 + s) for s in range(args.steps + args.warmup)]
    for s in range(args.warmup):
        oracle_rows_rate(v, t, rng_rows[s], x)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle_rows_rate(v, t, rng_rows[args.warmup + s], x)
    dt = time.perf_counter() - t0
    value = per_step * R * args.steps / dt      # entries of C X per second = unknowns*RHS/s
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64 complex)",
           "data": "synthetic", "config": {"workload": WORKLOAD, "nrhs": R, "parallelism": "host cores"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": "%d seeded rows of C per step times the %d columns, matrix-free dense "
                                      "Galerkin rows" % (per_step, R)},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------- replicas
def aggregate_ranks(ms, units_per_rank, dist=None, device="cpu"):
    """Replicas on N GPUs: the step time is the slowest rank's, the value is the units all
    ranks processed per second of that time (weak scaling)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return ms, world * units_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------------------- batched sweep
def _time_products(op, x, y, steps):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        op.matvec(x, out=y)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_batched(args):
    """Batched monostatic sweep on the cube-with-cylinder surface (~93k RWG, 186k unknowns):
    one product of C with args.batched plane-wave columns (phi in 2-degree steps at
    theta = 90 deg, right-hand sides of Eqs. 49-50 built by the oracle), FP32, with its error
    on sampled rows of the oracle's dense matrix.  Reported beside the main line."""
    import torch
    import oracle
    from paper_2210_04892_gb300 import bi
    from paper_2210_04892_gb300.inputs import SEED_BASE, cube_with_cylinder, sample_rows
    R = args.batched
    v, t = cube_with_cylinder()
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=R)
    info = op.info()
    ph = np.deg2rad(2.0 * np.arange(R))
    kh = -np.stack([np.cos(ph), np.sin(ph), 0 * ph], 1)
    pp = np.tile([0.0, 0.0, 1.0], (R, 1))
    xb = oracle.rhs_planewave(v, t, K0, 0, kh, pp)
    b = torch.from_numpy(xb.astype(np.complex64)).cuda()
    y = torch.empty_like(b)
    for _ in range(3):
        op.matvec(b, out=y)
    ms = _time_products(op, b, y, 20)
    stages = op.profile_stages(b, reps=5)
    yv = y.cpu().numpy().astype(np.complex128)
    # the same operator one column at a time (the plain one-RHS form)
    y1 = torch.empty_like(b[:1])
    b1 = b[:1].contiguous()
    for _ in range(3):
        op.matvec(b1, out=y1)
    ms1 = _time_products(op, b1, y1, 20)
    rows = sample_rows(op.n_unknowns, 64, seed=SEED_BASE + 12)
    _, _, err = oracle_rows_rate(v, t, rows, xb, yv)
    hbm, _ = peaks()
    tuned = op.tuned_config()
    out = {"workload": "cube 5 lambda + cylinder, %d RWG (%d unknowns), %d levels, FP32" %
                       (info["n_rwg"], info["n_unknowns"], info["levels"]),
           "nrhs": R, "ms_per_product": ms, "value": info["n_unknowns"] * R / (ms * 1e-3), "unit": UNIT,
           "one_rhs_value": info["n_unknowns"] / (ms1 * 1e-3), "setup_ms": info["setup_ms"],
           "rel_err_vs_oracle": err, "oracle_rows": len(rows),
           "stage_ms": stages, "stage_roofline": stage_roofline(info, R, stages, hbm),
           "tuned_config": tuned.strip().splitlines()}
    op.close()
    if args.sweep:
        out["sweep"] = run_sweep(v, t, R)
    return out


def run_sweep(v, t, R, n_inc=180, tol=1e-3):
    """The monostatic sweep end to end: 180 plane waves over phi (2-degree steps, theta = 90 deg,
    polarisation z), right-hand sides, GMRES solves and monostatic far fields on the GPU, in
    batches of R columns (64 + 64 + 52), against the same sweep one incidence at a time."""
    import torch
    from paper_2210_04892_gb300 import bi

    def sweep(op, batch, count=n_inc):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, sig = [], []
        for i0 in range(0, count, batch):
            ph = np.deg2rad(2.0 * np.arange(i0, min(count, i0 + batch)))
            kh = -np.stack([np.cos(ph), np.sin(ph), 0 * ph], 1)
            pp = np.tile([0.0, 0.0, 1.0], (len(ph), 1))
            b = op.rhs_planewave(kh, pp)
            x, it, rel = op.solve(b, tol=tol)
            F = op.farfield(x, -kh)                       # back-scatter directions of the batch
            diag = F[torch.arange(len(ph)), torch.arange(len(ph))]
            sig.append((4 * np.pi * (diag.abs() ** 2).sum(-1)).cpu().numpy())
            its.extend(int(i) for i in it)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return dt, its, np.concatenate(sig)

    ops = {}
    for batch in (R, 1):
        ops[batch] = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=batch, gmres_restart=30,
                                 gmres_maxit=300)
        sweep(ops[batch], batch, count=batch)  # warm-up: graph capture and autotuning
    dt_b, its_b, sig_b = sweep(ops[R], R)
    dt_1, its_1, sig_1 = sweep(ops[1], 1)
    for op in ops.values():
        op.close()
    return {"incidences": n_inc, "batch": R, "tol": tol, "seconds": dt_b, "gmres_iterations_mean": float(np.mean(its_b)),
            "one_at_a_time_seconds": dt_1, "one_at_a_time_iterations_mean": float(np.mean(its_1)),
            "monostatic_rcs_max_diff_db": float(np.max(np.abs(10 * np.log10(sig_b / sig_1)))),
            "form": "RHS + GMRES + monostatic far field per batch, FP32 products"}


# ---------------------------------------------------------------------------- serving stream
def _serve(bi, reqs, arrivals, tol, share=True, max_active=8):
    """Submit requests to a server at the given arrival times (s) and wait for all; returns
    per-request latency (s, arrival to solution), makespan (s), mean operator set-up ms, whether
    every request converged or reported, and the server's counters."""
    srv = bi.Server(max_active=max_active, share_operators=share)
    t0 = time.perf_counter()
    ids = []
    for q, ta in zip(reqs, arrivals):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0005)
        ids.append(srv.submit(q["verts"], q["tris"], q["k0"], q["khat"], q["phat"], tol=tol, op_mode=q["op_mode"]))
    lat, setup, ok = [], [], True
    for rid in ids:
        r = srv.wait(rid, timeout=3600)
        ok = ok and r["status"] in (bi.BI_OK, bi.BI_ERR_NOT_CONVERGED)
        lat.append(r["latency_ms"] / 1e3)
        setup.append(r["setup_ms"])
    makespan = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    built = [s for s in setup if s > 0]
    return np.array(lat), makespan, float(np.mean(built)) if built else 0.0, ok, stats


def _plain_fifo(bi, reqs, arrivals, tol):
    """The plain form: one request at a time in arrival order, its operator set up, then its
    right-hand sides solved one at a time (FP32, one-RHS products).  Each request's service time
    is measured; latencies follow from the arrivals of a single first-come-first-served server,
    and its capacity makespan (everything submitted at once) is the sum of the service times."""
    import torch
    service, ok = [], True
    for q in reqs:
        t0 = time.perf_counter()
        op = bi.Operator(q["verts"], q["tris"], q["k0"], precision="fp32", op_mode=q["op_mode"], max_rhs=1)
        for c in range(len(q["khat"])):
            b = op.rhs_planewave(q["khat"][c], q["phat"][c])
            x, its, rel = op.solve(b, tol=tol)
            ok = ok and bool(np.all(np.isfinite(rel)))
        torch.cuda.synchronize()
        op.close()
        service.append(time.perf_counter() - t0)
    finish, lat = 0.0, []
    for ta, sv in zip(arrivals, service):
        finish = max(finish, ta) + sv
        lat.append(finish - ta)
    return np.array(lat), finish - arrivals[0], ok, float(sum(service))


def run_serving(args):
    """Serving stream after c4 (request mix of inputs.serving_requests: spheres, ellipsoids and
    cubes, PEC or C block, plane waves; Poisson arrivals at 75% of the batched server's measured
    capacity): p50/p99 latency and solved unknowns*RHS per second of
      - the batched server (operators shared and cached, requests on one operator merged into
        one GMRES whose products are single batched launches),
      - the same server with one operator per request (requests overlap on the device but
        share no launch),
      - the plain form (one request at a time, one right-hand side at a time)."""
    from paper_2210_04892_gb300 import bi
    from paper_2210_04892_gb300.inputs import serving_requests
    reqs = serving_requests(args.serving, 2000, args.serving_max_unknowns, args.serving_max_rhs)
    tol = 1e-3
    work = sum((len(q["tris"]) * 3 // 2) * (2 if q["op_mode"] == 0 else 1) * len(q["khat"]) for q in reqs)
    n = len(reqs)
    _, span0, _, _, _ = _serve(bi, reqs, [0.0] * n, tol)
    span0_u = _serve(bi, reqs, [0.0] * n, tol, share=False)[1] if args.serving_unshared else None
    rate = 0.75 * n / span0
    rng = np.random.default_rng(20221011 + 31)
    arrivals = list(np.cumsum(rng.exponential(1.0 / rate, n)))
    arrivals = [a - arrivals[0] for a in arrivals]

    def summary(lat, span):
        return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "throughput": work / span}
    lat, span, setup_ms, ok, stats = _serve(bi, reqs, arrivals, tol)
    lat_u, span_u, setup_u, ok_u, stats_u = (_serve(bi, reqs, arrivals, tol, share=False) if args.serving_unshared
                                             else (None, None, None, True, None))
    lat_p, span_p, ok_p, cap_p = _plain_fifo(bi, reqs, arrivals, tol) if args.serving_plain else (None, None, True, None)
    out = {"requests": n, "unknowns_range": [2000, args.serving_max_unknowns], "max_rhs": args.serving_max_rhs,
           "distinct_operators": len({(q["shape"], len(q["tris"]), q["op_mode"]) for q in reqs}), "tol": tol,
           "arrival_rate_per_s": rate, "unit": "unknowns*RHS solved/s", "all_converged_or_reported": bool(ok and ok_u and ok_p),
           "capacity_makespan_s": span0, "capacity_throughput": work / span0,
           "note": "throughput under the Poisson stream is bounded by the arrivals (75% of the batched server's "
                   "capacity); capacity_throughput (every request submitted at once) compares the forms"}
    out.update(summary(lat, span))
    out.update({"mean_setup_ms": setup_ms, "server_stats": {k: v for k, v in stats.items() if k != "held_bytes"},
                "form": "operators shared and cached; requests on one operator merged into one batched GMRES"})
    if lat_u is not None:
        out["unshared"] = dict(summary(lat_u, span_u), mean_setup_ms=setup_u, capacity_makespan_s=span0_u,
                               capacity_throughput=work / span0_u,
                               form="one operator per request; requests overlap on the device, no shared launch")
    if lat_p is not None:
        out["plain"] = dict(summary(lat_p, span_p), capacity_makespan_s=cap_p, capacity_throughput=work / cap_p,
                            form="one request at a time (first come first served), one RHS at a time; latencies "
                                 "from each request's measured service time on the same arrivals")
    return out


# ---------------------------------------------------------------------------- GPU arm
def run_secondary(args, bi):
    """The 61,440-unknown sphere with one right-hand side (one product per step), with its
    roofline against the committed per-kernel DRAM summary and sampled oracle rows."""
    import torch
    from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, sample_rows
    v, t, meta = workload_mesh(SECONDARY["name"])
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=1)
    info = op.info()
    nun = op.n_unknowns
    x_np = complex_gaussian(nun, 1, seed=SEED_BASE + 1).astype(np.complex64)
    x = torch.from_numpy(x_np).cuda()
    y = torch.empty_like(x)
    for _ in range(20):
        op.matvec(x, out=y)
    ms = _time_products(op, x, y, 2000)
    stages = op.profile_stages(x, reps=50)
    hbm, kind = peaks()
    tr = measured_traffic()
    sr = stage_roofline(info, 1, stages, hbm)
    out = {"workload": SECONDARY["desc"], "n_unknowns": nun, "nrhs": 1, "ms_per_product": ms,
           "value": nun / (ms * 1e-3), "unit": UNIT, "stage_roofline": sr,
           "near_roofline": dict(sr["near"], traffic=tr.get("near", (None, None))[1],
                                 traffic_kernel=tr.get("near", (None, None))[0], peak_kind=kind)}
    if not args.no_cpu_baseline:
        rows = sample_rows(nun, 96, seed=SEED_BASE + 11)
        _, _, err = oracle_rows_rate(v, t, rows, x_np.astype(np.complex128), y.cpu().numpy().astype(np.complex128))
        out["rel_err_vs_oracle"] = err
    op.close()
    return out


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2210_04892_gb300 import bi
    from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, sample_rows
    v, t, meta = workload_mesh()
    R = HEADLINE["nrhs"]
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=R)
    info = op.info()
    nun = op.n_unknowns
    x_np = complex_gaussian(nun, R, seed=meta["seed"]).astype(np.complex64)
    x = torch.from_numpy(x_np).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        op.matvec(x, out=y)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        op.matvec(x, out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms, value = aggregate_ranks(ms, nun * R, dist, device="cuda")
    op.status()
    y_np = y.cpu().numpy()

    # end to end through the public host-buffer entry point (pinned host memory)
    xh = torch.from_numpy(x_np).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(3):
        op.matvec_host(xh, yh)
    n_e2e = max(5, min(args.steps, 20))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        op.matvec_host(xh, yh)
    t_e2e = (time.perf_counter() - t0) / n_e2e
    if dist:
        tt = torch.tensor([t_e2e], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    e2e = {"value": world * nun * R / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(xh.numel() * 8),
           "d2h_bytes_per_step": int(yh.numel() * 8), "ms_per_step": 1e3 * t_e2e}

    # live per-stage timing (serialised stages, CUDA events on the handle's stream)
    stages = op.profile_stages(x, reps=3)
    hbm, peak_kind = peaks()
    sr = stage_roofline(info, R, stages, hbm)
    dom = max((k for k in sr if k not in ("gather", "scatter")), key=lambda k: sr[k]["ms"])
    stages = {k: v for k, v in stages.items() if k in sr}
    tr = measured_traffic("dram_matvec_sphere_r20_3484860.md").get(dom)
    roofline = {"bound": sr[dom]["bound"], "kernel": dom, "achieved": sr[dom]["achieved"], "peak": sr[dom]["peak"],
                "unit": sr[dom]["unit"], "frac": sr[dom]["frac"],
                "peak_kind": peak_kind if sr[dom]["bound"] == "hbm" else "FP32 FMA peak from unit counts and clock",
                "traffic": tr[1] if tr else None, "traffic_kernel": tr[0] if tr else None,
                "algorithmic_bytes": sr[dom]["bytes"], "algorithmic_flops": sr[dom]["flops"],
                "stage_ms": stages, "stages": sr,
                "step_frac": sum(max(v["bytes"] / (hbm * 1e9), v["flops"] / (ALU_FP32_TFLOPS * 1e12))
                                 for v in sr.values()) / (ms * 1e-3)}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64 (fp32 complex)", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_unknowns": nun, "nrhs": R, "levels": info["levels"],
                      "near_pairs": info["near_pairs"], "parallelism": "replicas" if world > 1 else "single",
                      "l2": "inputs larger than L2 (near blocks + leaf patterns %.1f GB per step)" %
                            ((sr["near"]["bytes"] + sr["receive"]["bytes"]) / 1e9)},
           "roofline": roofline, "e2e": e2e, "clocks": clocks, "setup_ms": info["setup_ms"],
           "gpu_launches": launches_per_step(info, R, op.tuned_config()) * args.steps}
    out["rel_err_vs_oracle"] = golden_error(y_np)
    out["oracle_rows"] = "256 stored rows x 8 columns (tests/golden/c5_rows.json)"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        rows = sample_rows(nun, args.cpu_rows, seed=SEED_BASE + 11)
        rate, dt, err = oracle_rows_rate(v, t, rows, x_np.astype(np.complex128), y_np.astype(np.complex128))
        out["cpu_baseline"] = {"value": rate * R, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                               "sample": "%d seeded rows of C times the %d columns (matrix-free FP64 dense Galerkin "
                                         "rows), %.1f s" % (len(rows), R, dt)}
        if out["rel_err_vs_oracle"] is None:
            out["rel_err_vs_oracle"] = err
        out["rel_err_cpu_sample"] = err
    op.close()
    del x, y
    # the further sections are context for the headline: a failure in one is reported in its
    # place and does not cost the headline line
    for key, on, fn in (("secondary", args.secondary, lambda: run_secondary(args, bi)),
                        ("batched", args.batched, lambda: run_batched(args)),
                        ("serving", args.serving, lambda: run_serving(args))):
        if on and rank == 0:
            try:
                out[key] = fn()
            except Exception as e:  # noqa: BLE001 - any failure of a context section
                out[key] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
                print("bench: %s section failed: %r" % (key, e), file=sys.stderr, flush=True)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def profile_one(args):
    """One product of a workload between cudaProfilerStart and cudaProfilerStop, after set-up,
    tuning and warm-up products, so that ncu --profile-from-start off sees exactly one product."""
    import torch
    from paper_2210_04892_gb300 import bi
    from paper_2210_04892_gb300.inputs import SEED_BASE, complex_gaussian, cube_with_cylinder
    if args.profile_one == "cube_cylinder":
        v, t = cube_with_cylinder()
        R = args.nrhs or 8
    else:
        w = HEADLINE if args.profile_one == "headline" else SECONDARY
        v, t, _ = workload_mesh(w["name"])
        R = args.nrhs or w["nrhs"]
    op = bi.Operator(v, t, K0, digits=3, precision="fp32", op_mode=0, max_rhs=R)
    x = torch.from_numpy(complex_gaussian(op.n_unknowns, R, seed=SEED_BASE + 1).astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    for _ in range(max(3, args.warmup)):
        op.matvec(x, out=y)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    op.matvec(x, out=y)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    op.status()
    print(json.dumps({"profiled": args.profile_one, "n_unknowns": op.n_unknowns, "nrhs": R,
                      "tuned": op.tuned_config().strip().splitlines()}))
    op.close()


def main():
    args = parse()
    if args.profile_one:
        profile_one(args)
        return
    if args.serving_only:
        print(json.dumps({"serving": run_serving(args)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
