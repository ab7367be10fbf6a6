"""Benchmark: EGFEM Newton solves per second on the 1024 x 1024 triangulated unit square.

Workload (one "step"): a full Newton solve, from u0 = 0 to ||r|| <= 1e-10 ||r(u0)||, of
-div((1 + u^2) grad u) = f with u in P1 (1,050,625 nodes), w = u^2 in P2 (4,198,401
nodes), f manufactured from u = sin(pi x) sin(pi y), zero Dirichlet data.  Every step
runs the whole hot path in the CUDA library: the pointwise nonlinearity, the trilinear
tensor action (residual), the Jacobian fill, Jacobi-BiCGStab and the Newton update.

Reported (one JSON line on rank 0):
  value       FP64 Newton solves/s with inputs resident in HBM (CUDA events, max over ranks)
  e2e         the same through the public Python API with the load vector copied from
              pinned host memory and the solution copied back inside the timed region
  roofline    the dominant kernel (by share of the solve) against measured HBM bandwidth
  tensor_action  the fused tensor-action/Jacobian kernel against HBM and the FP64 pipe
  mixed       the same solve in mixed precision (FP32 operator/Krylov, FP64 residual)
  cpu_baseline   the FP64 CPU oracle on a bounded sample of the same workload

Inputs (operator ~0.5 GB, Jacobian ~0.1 GB) exceed the 129 MB L2, so no flush is needed
between timed steps.  --impl reference times the CPU oracle instead (the paper ships no
code; the oracle is the reference arm).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
SMS = 152                 # GB300 streaming multiprocessors
DFMA_PER_SM_CLK = 2       # FP64 FMAs per SM per clock on GB300 (nominal 1.25 TFLOP/s FP64)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def fp64_peak_tflops(peaks):
    """FP64 FMA peak from unit counts and the maximum SM clock: SMs x DFMA/clk x 2 flops x f."""
    return SMS * DFMA_PER_SM_CLK * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def roofline_of(k, hbm, peak_kind, fp64_peak):
    """Roofline of one profiled kernel: whichever of HBM bandwidth and (for FP64 kernels) the
    FP64 pipe it uses the larger fraction of is its bound."""
    sec = k["ms"] / 1e3
    gbs = k["bytes"] / sec / 1e9
    tf = k["flops"] / sec / 1e12
    # DRAM traffic needs ncu counters, which a timed run does not collect: null here; the ncu
    # captures of the kernels give it separately
    r = {"kernel": k["name"], "hbm_gbs": gbs, "hbm_frac": gbs / hbm,
         "hbm_peak_kind": f"{peak_kind} (hbm_gbs, copy)",
         "traffic": None, "bytes_per_launch": k["bytes"], "flops_per_launch": k["flops"]}
    if k["fp64"] and tf / fp64_peak > gbs / hbm:
        r.update({"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf / fp64_peak,
                  "peak_kind": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock"})
    else:
        r.update({"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                  "peak_kind": f"{peak_kind} (hbm_gbs, copy)"})
    if k["fp64"]:
        r["fp64_tflops"] = tf
        r["fp64_frac"] = tf / fp64_peak
    return r


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n):
    import workloads as wl
    mesh = wl.unit_square_mesh(n)
    cen = wl.cell_centroids(mesh)
    f_cell = wl.mms_source(cen[:, 0], cen[:, 1])
    return mesh, f_cell


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

class OracleSample:
    """The FP64 CPU oracle on a bounded sample of the n x n workload: a strip of `strip_rows`
    grid rows (set up once, untimed).  step() times the oracle's residual and Jacobian once and
    `kry_sample` BiCGStab iterations on the strip and returns (seconds the step took, the
    estimated seconds of one whole Newton solve): the strip's times scaled by (all nodes / strip
    nodes) and by the Newton and Krylov iteration counts of the solve being compared.  The
    BiCGStab loops run on the oracle's OpenMP threads (results independent of their number);
    the residual and Jacobian assembly are single-threaded."""

    def __init__(self, n, newton_steps, krylov_iters, strip_rows=64, kry_sample=60):
        import oracle
        import workloads as wl
        self.oracle = oracle
        full = wl.unit_square_mesh(n)
        keep = np.where(wl.cell_centroids(full)[:, 1] < strip_rows / n)[0]
        cells = full.cells[keep]
        nodes = np.unique(cells)
        remap = -np.ones(full.n_nodes, dtype=np.int64)
        remap[nodes] = np.arange(len(nodes))
        mesh = wl.Mesh(2, full.coords[nodes], remap[cells].astype(np.int32), full.dirichlet[nodes])
        self.P = oracle.Problem(mesh, a=("pow", 2.0), a_deg=2)
        cen = wl.cell_centroids(mesh)
        self.b = self.P.load_vector_cellwise(wl.mms_source(cen[:, 0], cen[:, 1])) * (1 - mesh.dirichlet)
        self.u = wl.random_vector(mesh.n_nodes, 1, 0.5) * (1 - mesh.dirichlet)
        self.scale = full.n_nodes / mesh.n_nodes
        self.newton_steps, self.krylov_iters, self.kry_sample = newton_steps, krylov_iters, kry_sample
        self.desc = (f"{strip_rows}-row strip of the {n}x{n} grid ({mesh.n_nodes} of {full.n_nodes} nodes): residual, "
                     f"Jacobian and {kry_sample} BiCGStab iterations timed per step, scaled by node count to "
                     f"{newton_steps} Newton steps and {krylov_iters} BiCGStab iterations per solve")

    def step(self, threads):
        self.oracle.set_threads(threads)
        t0 = time.perf_counter()
        self.P.residual(self.u, self.b, form="diff")
        J = self.P.jacobian(self.u)
        t1 = time.perf_counter()
        self.oracle.bicgstab(J, self.b, rtol=0.0, maxit=self.kry_sample)
        t2 = time.perf_counter()
        t_kry = (t2 - t1) / self.kry_sample
        per_solve = self.scale * ((self.newton_steps + 1) * (t1 - t0) + self.krylov_iters * t_kry)
        return t2 - t0, per_solve


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    # Newton/Krylov counts of the FP64 solve on this workload (the means of the library's timed
    # steps on the GPU)
    steps, kry = args.ref_newton_steps, args.ref_krylov_iters
    threads = os.cpu_count() or 1
    S = OracleSample(n, steps, kry)
    for _ in range(args.warmup):
        S.step(threads)
    secs, per = [], []
    for _ in range(args.steps):
        a, b = S.step(threads)
        secs.append(a)
        per.append(b)
    value = 1.0 / float(np.mean(per))
    line = {"impl": "reference", "metric": "newton_solves_per_s", "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"egfem_newton_2d_p1p2_u2_{n}x{n}", "grid": n, "w_space": "P2",
                       "newton_rtol": 1e-10, "parallelism": "replicas",
                       "step": "one bounded sample of the solve (see cpu_baseline.sample); value = solves/s "
                               "extrapolated from the samples"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "nproc": os.cpu_count(),
                             "kind": "oracle", "sample": S.desc},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def batched_adjoint_extra(torch, P, dev, count, n, barrier):
    """Solves + adjoint gradients per second on `count` instances of the n x n P1/P2
    u^2 problem with 16 x 16 cellwise sources theta_b (seed b) and j = 0.5 ||u - u_d||^2:
    the plain path (one FP64 handle, instances one after another) against the batched
    mixed path (one batch handle, batched Newton, block-diagonal adjoint)."""
    import workloads as wl
    from paper_2005_06193_gb300 import autograd as ag
    mesh = wl.unit_square_mesh(n)
    pc = torch.tensor(wl.param_cell_of_cells(mesh, 16), device=dev, dtype=torch.int64)
    ud = torch.tensor(wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1]), device=dev)
    free = torch.tensor(1.0 - mesh.dirichlet, device=dev)
    thetas = [torch.tensor(wl.adjoint_theta(b), device=dev) for b in range(count)]
    prob = P.make_problem(a=("pow", 2), a_degree=2)

    def grad_single(h, th):
        t = th.clone().requires_grad_(True)
        u = ag.newton_solve(ag.load_cellwise(t.reshape(-1)[pc], h), None, h)
        (0.5 * torch.sum(((u - ud) * free) ** 2)).backward()
        return t.grad

    hs = P.Handle(mesh, prob, P.default_options())
    grad_single(hs, thetas[0])   # warm
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_plain = [grad_single(hs, th) for th in thetas]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    hb = P.BatchHandle([mesh] * count, prob, P.default_options(precision=P.PREC_MIXED))
    off = hb.offsets

    def grad_batch():
        ts = [th.clone().requires_grad_(True) for th in thetas]
        d = ag.load_cellwise(torch.cat([t.reshape(-1)[pc] for t in ts]), hb)
        u = ag.newton_solve(d, None, hb)
        J = sum(0.5 * torch.sum(((u[off[b]:off[b] + mesh.n_nodes] - ud) * free) ** 2) for b in range(count))
        J.backward()
        return [t.grad for t in ts]

    grad_batch()   # warm (includes the tile autotuning)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_batch = grad_batch()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    err = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(g_batch, g_plain))
    tbytes, tshare = hb.tensor_storage()
    hs.close()
    hb.close()
    return {"workload": f"{count} x {n}x{n} P1/P2 u^2, 16x16 cellwise theta, j = 0.5||u-u_d||^2",
            "unit": "solves+gradients/s", "plain_fp64_sequential": count / t_plain, "batched_mixed": count / t_batch,
            "speedup": t_plain / t_batch, "max_rel_gradient_difference": err,
            "tensor_bytes": tbytes, "tensor_shared_by": tshare}


def p3_instances(count):
    """The first `count` of the 256 seeded instances (n ~ U{64..512}, w = u^3 in P3, 8-mode sine
    sources): meshes, the problem and the cellwise sources."""
    import workloads as wl
    inst = wl.batch_instances(count=256, seed=0)[:count]
    meshes = [wl.unit_square_mesh(n) for n, _ in inst]
    fs = []
    for (n, src), mesh in zip(inst, meshes):
        cen = wl.cell_centroids(mesh)
        fs.append(src(cen[:, 0], cen[:, 1]))
    return meshes, fs


def p3_batch(torch, P, dev, meshes, fs, **opts):
    prob = P.make_problem(a=("pow", 3), a_degree=3)
    hb = P.BatchHandle(meshes, prob, P.default_options(**{"precision": P.PREC_MIXED, **opts}))
    d = torch.empty(hb.sizes.n_nodes, device=dev, dtype=torch.float64)
    hb.load_cellwise(torch.tensor(np.concatenate(fs), device=dev), d)
    return hb, d


def profile_batch(torch, P, dev, count=16):
    """One batched Newton step (host loop, BiCGStab run for exactly 40 iterations: a fixed forcing
    term of 1e-14) on the first `count` P3 instances, twice; the second call, after the tile
    autotuning, runs inside the NVTX range "capture" (ncu --nvtx --nvtx-include capture/ selects
    its batched solve)."""
    meshes, fs = p3_instances(count)
    hb, d = p3_batch(torch, P, dev, meshes, fs, newton_graph=0, newton_maxit=1, newton_rtol=0.9, krylov_maxit=40,
                     fixed_eta=1, eta_max=1e-14)
    u = torch.zeros_like(d)
    hb.batch_newton_solve(u, d, check=False)
    torch.cuda.synchronize()
    u.zero_()
    torch.cuda.nvtx.range_push("capture")
    st = hb.batch_newton_solve(u, d, check=False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    out = {"instances": count, "rows": int(hb.sizes.n_nodes), "krylov_iters": [int(s.krylov_iters) for s in st],
           "status": [int(s.status) for s in st]}
    hb.close()
    return out


def profile_adjbatch(torch, P, dev, count=16, n=512, fp64=False):
    """One batched Newton step (host loop, exactly 40 BiCGStab iterations: a fixed forcing term of
    1e-14; mixed precision, or FP64 with fp64) on `count` instances of the n x n P1/P2 u^2 problem on ONE mesh (the adjoint workload's
    layout: the tensor stored once for all instances), with seeded random loads, twice; the second
    call's batched solve is the one to capture (ncu -s 1 -c 1 on pkwb_solve)."""
    import workloads as wl
    mesh = wl.unit_square_mesh(n)
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    hb = P.BatchHandle([mesh] * count, prob, P.default_options(
        precision=P.PREC_FP64 if fp64 else P.PREC_MIXED, newton_graph=0, newton_maxit=1, newton_rtol=0.9,
        krylov_maxit=40, fixed_eta=1, eta_max=1e-14))
    free = 1 - mesh.dirichlet
    d = hb.scatter([wl.random_vector(mesh.n_nodes, 3 + b, 1.0) * free for b in range(count)])
    for _ in range(2):
        u = torch.zeros_like(d)
        st = hb.batch_newton_solve(u, d, check=False)
        torch.cuda.synchronize()
    out = {"instances": count, "rows": int(hb.sizes.n_nodes), "tensor_storage": hb.tensor_storage(),
           "krylov_iters": [int(s.krylov_iters) for s in st][:4]}
    hb.close()
    return out


def profile_adjoint64(torch, P, dev, count, n):
    """The batched half of the adjoint workload (count instances of the n x n P1/P2 u^2 problem on
    one mesh, 16 x 16 cellwise theta, j = 0.5 ||u - u_d||^2): the batched mixed Newton solve and the
    block-diagonal adjoint through autograd, a warm pass and one more (for an ncu launch list)."""
    import workloads as wl
    from paper_2005_06193_gb300 import autograd as ag
    mesh = wl.unit_square_mesh(n)
    pc = torch.tensor(wl.param_cell_of_cells(mesh, 16), device=dev, dtype=torch.int64)
    ud = torch.tensor(wl.adjoint_target()(mesh.coords[:, 0], mesh.coords[:, 1]), device=dev)
    free = torch.tensor(1.0 - mesh.dirichlet, device=dev)
    thetas = [torch.tensor(wl.adjoint_theta(b), device=dev) for b in range(count)]
    hb = P.BatchHandle([mesh] * count, P.make_problem(a=("pow", 2), a_degree=2),
                       P.default_options(precision=P.PREC_MIXED, newton_graph=0))
    off = hb.offsets
    for _ in range(2):
        ts = [th.clone().requires_grad_(True) for th in thetas]
        d = ag.load_cellwise(torch.cat([t.reshape(-1)[pc] for t in ts]), hb)
        u = ag.newton_solve(d, None, hb)
        J = sum(0.5 * torch.sum(((u[off[b]:off[b] + mesh.n_nodes] - ud) * free) ** 2) for b in range(count))
        t0 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
    out = {"instances": count, "rows": int(hb.sizes.n_nodes), "tensor_storage": hb.tensor_storage(),
           "backward_s": time.perf_counter() - t0}
    hb.close()
    return out


def profile_p3batch(torch, P, dev, count):
    """The batched mixed Newton solve of `count` P3 instances (the default 256) with the host
    Newton loop, so that every kernel is a top-level launch (for an ncu launch list): a warm
    solve, then one more."""
    meshes, fs = p3_instances(count)
    hb, d = p3_batch(torch, P, dev, meshes, fs, newton_graph=0)
    u = torch.zeros_like(d)
    hb.batch_newton_solve(u, d)
    u.zero_()
    t0 = time.perf_counter()
    st = hb.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    out = {"instances": count, "rows": int(hb.sizes.n_nodes), "seconds": time.perf_counter() - t0,
           "krylov_iters_sum": int(sum(s.krylov_iters for s in st)), "newton_max": int(max(s.newton_iters for s in st))}
    hb.close()
    return out


def batched_p3_extra(torch, P, dev, count, barrier):
    """Newton solves per second on the first `count` instances of the 256-instance batch
    (n ~ U{64..512}, w = u^3 in P3, 8-mode sine sources): plain sequential FP64 solves
    against one batched mixed solve."""
    meshes, fs = p3_instances(count)
    prob = P.make_problem(a=("pow", 3), a_degree=3)
    hb, d = p3_batch(torch, P, dev, meshes, fs)
    u = torch.zeros_like(d)
    hb.batch_newton_solve(u, d)   # warm + tile autotuning
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u.zero_()
    st = hb.batch_newton_solve(u, d)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    ok = all(s.status == 0 and s.res_final <= 1e-10 * s.res0 for s in st)
    t_plain = 0.0
    for mesh, f in zip(meshes, fs):
        h = P.Handle(mesh, prob, P.default_options())
        db = torch.empty(mesh.n_nodes, device=dev, dtype=torch.float64)
        h.load_cellwise(torch.tensor(f, device=dev), db)
        ub = torch.zeros_like(db)
        h.newton_solve(ub, db)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ub.zero_()
        h.newton_solve(ub, db)
        torch.cuda.synchronize()
        t_plain += time.perf_counter() - t0
        h.close()
    hb.close()
    return {"workload": (f"the 256 seeded instances, n in [64, 512], P1/P3 u^3" if count == 256 else
                         f"first {count} of the 256 seeded instances, n in [64, 512], P1/P3 u^3"),
            "unit": "solves/s", "plain_fp64_sequential": count / t_plain, "batched_mixed": count / t_batch,
            "speedup": t_plain / t_batch, "all_converged_1e-10": ok,
            "rows": int(hb.sizes.n_nodes)}


def _mf_kernel_line(prof, hbm, fp64_peak):
    pm = next(p for p in prof if p["name"].startswith("tensor_action"))
    return {"kernel": "mf_cell_kernel + mf_row_kernel", "ms": pm["ms"], "bytes_per_launch": pm["bytes"],
            "achieved_gbs": pm["bytes"] / (pm["ms"] / 1e3) / 1e9, "frac_hbm": pm["bytes"] / (pm["ms"] / 1e3) / 1e9 / hbm,
            "fp64_tflops": pm["flops"] / (pm["ms"] / 1e3) / 1e12,
            "fp64_frac_of_peak": pm["flops"] / (pm["ms"] / 1e3) / 1e12 / fp64_peak}


def gradient_setup(torch, P, dev, n):
    """Minimal surface on the n x n square (Sec. 5): a = (1 + |grad u|^2)^(-1/2) on W = P0,
    u_D = x y (x + y), manufactured source sampled at cell centroids, Newton from the boundary
    data with a smooth interior bump.  Returns (handle, d, u0)."""
    import workloads as wl
    mesh = wl.unit_square_mesh(n)
    h = P.Handle(mesh, P.make_problem(a=("gradpow", -0.5, 1.0), a_degree=0, kappa=0.0),
                 P.default_options(op=P.OP_MATRIX_FREE))
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    ue = wl.minsurf_exact(x, y)
    xc = wl.cell_centroids(mesh)
    f = torch.tensor(wl.minsurf_source(xc[:, 0], xc[:, 1]), device=dev, dtype=torch.float64)
    d = torch.empty(mesh.n_nodes, device=dev, dtype=torch.float64)
    h.load_cellwise(f, d)
    d += torch.tensor(ue * mesh.dirichlet, device=dev)
    u0 = torch.tensor(ue + 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y), device=dev, dtype=torch.float64)
    return h, d, u0


def quadrature_setup(torch, P, dev, n):
    """The quadratic example -lap u + u^2 = d on the n x n square (Sec. 5) with W_c = I_3 (the
    paper's Case 3 choice for it), u_D = x y (x + y), manufactured source at cell centroids,
    Newton from the boundary data.  Returns (handle, d, u0)."""
    import workloads as wl
    mesh = wl.unit_square_mesh(n)
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, kappa=1.0, c=("pow", 2), c_degree=3, c_space="quad",
                                      gamma=1.0), P.default_options(op=P.OP_MATRIX_FREE))
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    uD = wl.minsurf_exact(x, y) * mesh.dirichlet
    xc = wl.cell_centroids(mesh)
    f = torch.tensor(wl.quadratic_source(xc[:, 0], xc[:, 1]), device=dev, dtype=torch.float64)
    d = torch.empty(mesh.n_nodes, device=dev, dtype=torch.float64)
    h.load_cellwise(f, d)
    d += torch.tensor(uD, device=dev)
    return h, d, torch.tensor(uD, device=dev, dtype=torch.float64)


# Table 1 (Sec. 5, superconductivity, decompositions (a), (b)): the paper's own solve times in seconds
# (Matlab R2019b on an i7-8700, Picard iteration) for context only; None where its Picard
# iteration did not converge
TABLE1_SECONDS = {("b", "p3", 1.0): 0.076, ("b", "i4", 1.0): 0.077, ("b", "p3", 1e-2): 0.599,
                  ("b", "i4", 1e-2): 0.579, ("b", "p3", 1e-3): None, ("b", "i4", 1e-3): None,
                  ("a", "p2", 1.0): 0.146, ("a", "i4", 1.0): 0.182, ("a", "p2", 1e-2): 0.577,
                  ("a", "i4", 1e-2): 0.702, ("a", "p2", 1e-3): 1.185, ("a", "i4", 1e-3): 1.425}


def supercond_setup(torch, P, dev, n, nu, space, decomp="b"):
    """Superconductivity example on the n x n square (Sec. 5), decomposition (b): nu K u + M u +
    M^c c with c = u^3 on W_c = P3 or I_4; or (a): nu K u + M3 : (u x c~), c~ = u^2 + 1, written as
    sigma M u plus the product reaction with c = u^2 on W_c = P2 or I_4.  u_D = sin(2 pi x)
    sin(2 pi y) e^(2x) / 6, manufactured source at cell centroids, Newton from the boundary data.
    Returns (handle, d, u0)."""
    import workloads as wl
    mesh = wl.unit_square_mesh(n)
    deg, cs = {"p3": (3, "lagrange"), "p2": (2, "lagrange"), "i4": (4, "quad")}[space]
    h = P.Handle(mesh, P.make_problem(a=None, a_degree=1, kappa=nu, c=("pow", 2 if decomp == "a" else 3), c_degree=deg,
                                      c_space=cs, gamma=1.0, sigma=1.0, c_product=decomp == "a"),
                 P.default_options(op=P.OP_MATRIX_FREE, newton_maxit=100))
    x, y = mesh.coords[:, 0], mesh.coords[:, 1]
    uD = wl.supercond_exact(x, y) * mesh.dirichlet
    xc = wl.cell_centroids(mesh)
    f = torch.tensor(wl.supercond_source(xc[:, 0], xc[:, 1], nu), device=dev, dtype=torch.float64)
    d = torch.empty(mesh.n_nodes, device=dev, dtype=torch.float64)
    h.load_cellwise(f, d)
    d += torch.tensor(uD, device=dev)
    return h, d, torch.tensor(uD, device=dev, dtype=torch.float64)


def supercond_extra(torch, P, dev, steps, barrier, hbm, fp64_peak, n_big):
    rows = []
    cases = [(dec, sp, nu) for dec, sps in (("a", ("p2", "i4")), ("b", ("p3", "i4"))) for nu in (1.0, 1e-2, 1e-3)
             for sp in sps]
    for decomp, space, nu in cases:
        h, d, u0 = supercond_setup(torch, P, dev, 64, nu, space, decomp)
        u = u0.clone()
        h.newton_solve(u, d)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(steps, 5)
        e0.record()
        for _ in range(reps):
            u.copy_(u0)
            st = h.newton_solve(u, d)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        rows.append({"decomposition": decomp, "nu": nu, "w_c": space, "unknowns": h.sizes.n_nodes + h.sizes.n_wc,
                     "solves_per_s": 1e3 / ms, "ms_per_solve": ms, "newton_iters": st.newton_iters,
                     "krylov_iters": int(st.krylov_iters), "status": int(st.status),
                     "paper_seconds_context": TABLE1_SECONDS[(decomp, space, nu)]})
        h.close()
    out = {"workload": "superconductivity decompositions (a) and (b), 64x64 grid (Table 1), Newton to 1e-10",
           "table1": rows}
    if n_big:
        out["large"] = next_row_extra(torch, P, dev, n_big, min(steps, 3), barrier,
                                      lambda t, PP, dv, n: supercond_setup(t, PP, dv, n, 1.0, "p3"),
                                      f"superconductivity_b_p3_nu1_{n_big}x{n_big}", hbm, fp64_peak)
    return out


def bratu_extra(torch, P, dev, steps, barrier, hbm, fp64_peak, n=64):
    """Bratu -lap u = 2 e^u on the n^3 cube (6 Kuhn tetrahedra per cube; e^u interpolated in P1,
    GFEM), f = 0, Newton from 0: FP64 and mixed (FP32 operator and Krylov, FP64 residual)
    solves, the mixed error against the FP64 solution, and each path's tensor action."""
    import workloads as wl
    mesh = wl.unit_cube_mesh(n)
    prob = P.make_problem(a=None, a_degree=1, c=("exp",), c_degree=1, gamma=-2.0)
    d = torch.zeros(mesh.n_nodes, device=dev, dtype=torch.float64)
    out, sols = {"workload": f"bratu_3d_{n}^3_gfem_p1", "n_nodes": mesh.n_nodes, "n_cells": mesh.n_cells}, {}
    for prec in ("fp64", "mixed"):
        h = P.Handle(mesh, prob, P.default_options(precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64))
        u = torch.zeros_like(d)
        h.newton_solve(u, d)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            u.zero_()
            st = h.newton_solve(u, d)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = h.profile_kernels(u, d, reps=20)
        ta = next(p for p in prof if p["name"] in ("csf_fused", "csf_mixed"))
        out[prec] = {"value": 1e3 / ms, "unit": "solves/s", "ms_per_step": ms, "newton_iters": st.newton_iters,
                     "krylov_iters": int(st.krylov_iters), "final_rel_residual": st.res_final / st.res0,
                     "tensor_action": {"kernel": ta["name"], "ms": ta["ms"],
                                       "achieved_gbs": ta["bytes"] / (ta["ms"] / 1e3) / 1e9,
                                       "frac_hbm": ta["bytes"] / (ta["ms"] / 1e3) / 1e9 / hbm}}
        sols[prec] = u.clone()
        h.close()
    out["mixed_rel_error_vs_fp64"] = float(torch.linalg.norm(sols["mixed"] - sols["fp64"]) / torch.linalg.norm(sols["fp64"]))
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


def next_row_extra(torch, P, dev, n, steps, barrier, setup, workload, hbm, fp64_peak):
    h, d, u0 = setup(torch, P, dev, n)
    u = u0.clone()
    h.newton_solve(u, d)
    torch.cuda.synchronize()
    stats = []
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        u.copy_(u0)
        stats.append(h.newton_solve(u, d))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = stats[-1]
    prof = h.profile_kernels(u, d, reps=20)
    out = {"workload": workload, "value": steps / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms / steps,
           "newton_iters": st.newton_iters, "krylov_iters": int(st.krylov_iters),
           "final_rel_residual": st.res_final / st.res0, "gpu_launches": int(sum(s.kernel_launches for s in stats)),
           "n_wa": h.sizes.n_wa, "n_wc": h.sizes.n_wc,
           "tensor_action": _mf_kernel_line(prof, hbm, fp64_peak),
           "kernels": [{"name": p["name"], "ms": p["ms"]} for p in prof]}
    h.close()
    return out


def latency_c1(torch, P, dev, reps, barrier, n=32):
    """The 32 x 32 workload (1089 P1, 4225 P2 nodes; the whole problem sits in L2): FP64 Newton
    solves per second with the library's defaults (one-cluster BiCGStab, graph-resident Newton
    loop), same source and target as the 1024 x 1024 line."""
    mesh, f_cell = make_workload(n)
    h = P.Handle(mesh, P.make_problem(a=("pow", 2), a_degree=2), P.default_options())
    f = torch.tensor(f_cell, device=dev, dtype=torch.float64)
    d = torch.empty(mesh.n_nodes, device=dev, dtype=torch.float64)
    h.load_cellwise(f, d)
    u = torch.zeros_like(d)
    for _ in range(3):
        u.zero_()
        h.newton_solve(u, d)
    ms, stats = timed_solves(torch, h, [d], u, reps, barrier)
    st = stats[-1]
    out = {"workload": f"egfem_newton_2d_p1p2_u2_{n}x{n}", "value": reps / (ms / 1e3), "unit": "solves/s",
           "ms_per_step": ms / reps, **mean_iters(stats), "final_rel_residual": st.res_final / st.res0,
           "krylov_driver": "cluster" if h.options.krylov_cluster >= 0 else "grid", "newton_loop": "graph"}
    h.close()
    return out


def whole_job_rate(dist, world, units, ms, device):
    """Units per second for the whole job: every rank's `units` over the slowest rank's time
    (`ms` is this rank's time; the maximum over ranks is taken with an all-reduce).  Returns
    (rate, slowest ms)."""
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * units / (ms_max / 1e3), ms_max


def perturbed_loads(d, count):
    """count copies of the load vector d scaled by 1 + k 2^-44 (k = 0 .. count-1): the same
    workload to about 13 digits.  The BiCGStab iteration count of a solve moves by up to about
    20 % under such perturbations (rounding decides when the erratic residual history crosses
    its tolerance), so each timed step solves its own copy and the rate reflects the mean count
    rather than one draw."""
    return [d * (1.0 + k * 2.0 ** -44) for k in range(count)]


def mean_iters(stats):
    k = [int(s.krylov_iters) for s in stats]
    return {"krylov_iters": round(sum(k) / len(k), 1), "krylov_iters_range": [min(k), max(k)],
            "newton_iters": round(sum(s.newton_iters for s in stats) / len(stats), 2)}


def timed_solves(torch, h, ds, u, steps, rank_barrier):
    """steps Newton solves from u = 0, step i on the load vector ds[i % len(ds)]"""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    rank_barrier()
    torch.cuda.synchronize()
    ev0.record()
    for i in range(steps):
        u.zero_()
        stats.append(h.newton_solve(u, ds[i % len(ds)]))
    ev1.record()
    torch.cuda.synchronize()
    rank_barrier()
    return ev0.elapsed_time(ev1), stats


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-mf", action="store_true")
    ap.add_argument("--no-picard", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-next", action="store_true", help="skip the gradient-coefficient and I_k lines")
    ap.add_argument("--no-bratu", action="store_true", help="skip the 64^3 Bratu line")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--p3-instances", type=int, default=256)
    ap.add_argument("--ref-newton-steps", type=int, default=7)
    ap.add_argument("--ref-krylov-iters", type=int, default=2935)
    ap.add_argument("--profile-only", default=None,
                    choices=["fp64", "mixed", "gradient", "quadrature", "supercond", "batch", "p3batch", "adjbatch",
                             "adjbatch64", "adjoint64"],
                    help="build the workload (gradient: minimal surface; quadrature: quadratic example with I_3), "
                         "run the per-kernel profile once and print it (for ncu captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2005_06193_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    if args.profile_only == "batch":
        print(json.dumps(profile_batch(torch, P, torch.device("cuda", local))), flush=True)
        return
    if args.profile_only in ("adjbatch", "adjbatch64"):
        print(json.dumps(profile_adjbatch(torch, P, torch.device("cuda", local), fp64=args.profile_only == "adjbatch64")),
              flush=True)
        return
    if args.profile_only == "adjoint64":
        print(json.dumps(profile_adjoint64(torch, P, torch.device("cuda", local), args.batch_instances, args.batch_n)),
              flush=True)
        return
    if args.profile_only == "p3batch":
        print(json.dumps(profile_p3batch(torch, P, torch.device("cuda", local), args.p3_instances)), flush=True)
        return
    if args.profile_only in ("gradient", "quadrature", "supercond"):
        setup = {"gradient": gradient_setup, "quadrature": quadrature_setup,
                 "supercond": lambda t, PP, dv, n: supercond_setup(t, PP, dv, n, 1.0, "p3")}[args.profile_only]
        hp, d, u0 = setup(torch, P, torch.device("cuda", local), args.n)
        print(json.dumps(hp.profile_kernels(u0, d, reps=1)), flush=True)
        hp.close()
        return
    mesh, f_cell = make_workload(args.n)
    prob = P.make_problem(a=("pow", 2), a_degree=2)
    if args.profile_only:
        hp = P.Handle(mesh, prob, P.default_options(precision=P.PREC_MIXED if args.profile_only == "mixed" else P.PREC_FP64))
        f = torch.tensor(f_cell, device="cuda", dtype=torch.float64)
        d = torch.empty(mesh.n_nodes, device="cuda", dtype=torch.float64)
        hp.load_cellwise(f, d)
        # a seeded state with the converged solution's scale (|u| up to about 0.3), zero on the
        # Dirichlet rows: the kernels' work does not depend on u, their instruction paths a little
        import workloads as wl
        u = torch.tensor(wl.random_vector(mesh.n_nodes, 5, 0.3) * (1 - mesh.dirichlet), device="cuda")
        print(json.dumps(hp.profile_kernels(u, d, reps=1)), flush=True)
        hp.close()
        return
    # the host Newton loop (newton_graph = 0): at this size it is as fast as the graph-resident
    # loop (timed below), and ncu sees every kernel of it (not those inside a conditional node)
    h = P.Handle(mesh, prob, P.default_options(newton_graph=0))
    dev = torch.device("cuda", local)
    f = torch.tensor(f_cell, device=dev, dtype=torch.float64)
    d = torch.empty(mesh.n_nodes, device=dev, dtype=torch.float64)
    h.load_cellwise(f, d)
    ds = perturbed_loads(d, args.steps)
    u = torch.zeros(mesh.n_nodes, device=dev, dtype=torch.float64)
    for i in range(args.warmup):
        u.zero_()
        h.newton_solve(u, ds[i % len(ds)])
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, stats = timed_solves(torch, h, ds, u, args.steps, barrier)
    clocks = clk.summary()
    value, ms_max = whole_job_rate(dist, world, args.steps, ms, dev)
    st = stats[-1]
    its = mean_iters(stats)
    launches = int(sum(s.kernel_launches for s in stats))

    # end to end through the public API with host buffers
    d_hosts = [x.cpu().pin_memory() for x in ds]
    u_host = torch.empty(mesh.n_nodes, dtype=torch.float64).pin_memory()
    d_dev = torch.empty_like(d)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        d_dev.copy_(d_hosts[i % len(d_hosts)], non_blocking=True)
        u.zero_()
        h.newton_solve(u, d_dev)
        u_host.copy_(u, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value, _ = whole_job_rate(dist, world, args.steps, e2e_ms, dev)

    # per-kernel profile at the converged state (CUDA events on the library's stream)
    prof = h.profile_kernels(u, d, reps=20)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    fp64_peak = fp64_peak_tflops(peaks)
    counts = {"csf_fused": its["newton_iters"] + 1}
    for k in ("kry_v", "kry_s", "kry_t", "kry_x", "kry_p", "kry_persistent", "kry_window", "kry_cluster"):
        counts[k] = its["krylov_iters"]
    share = {p["name"]: p["ms"] * counts.get(p["name"], 0) for p in prof}
    total_share = sum(share.values())
    dom = max(prof, key=lambda p: share[p["name"]])
    roofline = roofline_of(dom, hbm, peak_kind, fp64_peak)
    roofline["share_of_solve"] = share[dom["name"]] / (ms_max / args.steps)
    if dom["name"] in ("kry_persistent", "kry_window", "kry_cluster"):
        roofline["units_per_launch"] = f"one launch runs a whole BiCGStab solve; ms and bytes are per iteration"
    csf = next(p for p in prof if p["name"] == "csf_fused")
    # second half of the metric: the tensor action (nodal pass + fused residual / Jacobian fill)
    # against HBM, with the FP64 pipe (its binding unit) beside it
    ta_gbs = csf["bytes"] / (csf["ms"] / 1e3) / 1e9
    ta_tf = csf["flops"] / (csf["ms"] / 1e3) / 1e12
    roofline_ta = {"kernel": "wnode_kernel + csf_fused_kernel (residual + Jacobian fill, FP64)", "bound": "hbm",
                   "achieved": ta_gbs, "peak": hbm, "unit": "GB/s", "frac": ta_gbs / hbm, "traffic": None,
                   "peak_kind": f"{peak_kind} (hbm_gbs, copy)", "bytes_per_launch": csf["bytes"], "ms": csf["ms"],
                   "fp64_tflops": ta_tf, "fp64_frac": ta_tf / fp64_peak,
                   "fp64_peak_kind": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock"}
    tensor_action = {"kernel": "csf_fused", "ms": csf["ms"], "achieved_gbs": csf["bytes"] / (csf["ms"] / 1e3) / 1e9,
                     "frac_hbm": csf["bytes"] / (csf["ms"] / 1e3) / 1e9 / hbm,
                     "fp64_tflops": csf["flops"] / (csf["ms"] / 1e3) / 1e12,
                     "fp64_frac_of_peak": csf["flops"] / (csf["ms"] / 1e3) / 1e12 / fp64_peak,
                     "bytes_per_launch": csf["bytes"]}

    # the same FP64 solve with the graph-captured iteration kernels instead of the persistent solve
    hg = P.Handle(mesh, prob, P.default_options(krylov_persistent=0))
    u.zero_()
    hg.newton_solve(u, d)
    msg, sg = timed_solves(torch, hg, ds, u, min(args.steps, 3), barrier)
    graph_driver = {"value": world * min(args.steps, 3) / (msg / 1e3), "unit": "solves/s",
                    "ms_per_step": msg / min(args.steps, 3), **mean_iters(sg),
                    "gpu_launches_per_solve": int(sg[-1].kernel_launches)}
    hg.close()

    out = {"metric": "newton_solves_per_s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"egfem_newton_2d_p1p2_u2_{args.n}x{args.n}", "grid": args.n, "n_p1": mesh.n_nodes,
                      "n_p2": h.sizes.n_wa, "newton_rtol": 1e-10, "precision": "fp64", "operator": "csf",
                      "parallelism": "replicas" if world > 1 else "single", "l2": "inputs larger than L2 (no flush)",
                      "krylov_driver": "persistent" if h.options.krylov_persistent else "graph",
                      "newton_loop": "host",
                      "rhs": "step k solves with the load vector scaled by 1 + k 2^-44 (the iteration count's "
                             "sensitivity to rounding averaged over the steps)"},
           **its,
           "final_rel_residual": st.res_final / st.res0,
           "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * mesh.n_nodes,
                   "d2h_bytes_per_step": 8 * mesh.n_nodes},
           "gpu_launches": launches, "roofline": roofline, "roofline_tensor_action": roofline_ta,
           "tensor_action": tensor_action, "clocks": clocks,
           "kernels": [{**p, "share": share[p["name"]] / total_share} for p in prof],
           "fp64_graph_driver": graph_driver}

    # the same FP64 solve with the graph-resident Newton loop (the library's default)
    hgl = P.Handle(mesh, prob, P.default_options())
    u.zero_()
    hgl.newton_solve(u, d)
    msl, sgl = timed_solves(torch, hgl, ds, u, args.steps, barrier)
    out["graph_newton_loop"] = {"value": world * args.steps / (msl / 1e3), "unit": "solves/s",
                                "ms_per_step": msl / args.steps, **mean_iters(sgl),
                                "gpu_launches_per_solve": int(sgl[-1].kernel_launches)}
    hgl.close()

    out["latency_32x32"] = latency_c1(torch, P, dev, max(args.steps, 20), barrier)

    if not args.no_mixed:
        hm = P.Handle(mesh, prob, P.default_options(precision=P.PREC_MIXED, newton_graph=0))
        for i in range(max(1, args.warmup)):
            u.zero_()
            hm.newton_solve(u, ds[i % len(ds)])
        msm, sm = timed_solves(torch, hm, ds, u, args.steps, barrier)
        sl = sm[-1]
        mprof = hm.profile_kernels(u, d, reps=20)
        out["mixed"] = {"value": world * args.steps / (msm / 1e3), "unit": "solves/s", "ms_per_step": msm / args.steps,
                        **mean_iters(sm), "final_rel_residual": sl.res_final / sl.res0,
                        "speedup_vs_fp64": (ms_max / msm), "fp64_rescues": int(sum(x.fp64_rescues for x in sm)),
                        "kernels": [{"name": p["name"], "ms": p["ms"], "gbs": p["bytes"] / (p["ms"] / 1e3) / 1e9,
                                     "frac_hbm": p["bytes"] / (p["ms"] / 1e3) / 1e9 / hbm} for p in mprof]}
        out["mixed"]["gpu_launches"] = int(sum(s.kernel_launches for s in sm))
        cm = next((p for p in mprof if p["name"] == "csf_mixed"), None)
        if cm is not None:
            out["tensor_action_mixed"] = {
                "kernel": "wnode_kernel + csf_mixed_kernel (FP64 residual, FP32 Jacobian)", "ms": cm["ms"],
                "achieved_gbs": cm["bytes"] / (cm["ms"] / 1e3) / 1e9, "frac_hbm": cm["bytes"] / (cm["ms"] / 1e3) / 1e9 / hbm,
                "fp64_tflops": cm["flops"] / (cm["ms"] / 1e3) / 1e12, "bytes_per_launch": cm["bytes"],
                "speedup_vs_fp64": csf["ms"] / cm["ms"]}
        hm.close()

    if not args.no_picard:
        # the paper's own iteration (Picard, frozen coefficient) on the same workload
        hpi = P.Handle(mesh, prob, P.default_options(iteration=P.ITER_PICARD, newton_maxit=200))
        u.zero_()
        hpi.newton_solve(u, d)
        msp, spi = timed_solves(torch, hpi, ds, u, min(args.steps, 2), barrier)
        sl = spi[-1]
        out["picard"] = {"value": world * min(args.steps, 2) / (msp / 1e3), "unit": "solves/s",
                         "ms_per_step": msp / min(args.steps, 2), "picard_iters": sl.newton_iters,
                         "krylov_iters": int(sl.krylov_iters), "final_rel_residual": sl.res_final / sl.res0,
                         "time_vs_newton": (msp / min(args.steps, 2)) / (ms_max / args.steps)}
        hpi.close()

    if not args.no_mf:
        hmf = P.Handle(mesh, prob, P.default_options(op=P.OP_MATRIX_FREE))
        pm = next(p for p in hmf.profile_kernels(u, d, reps=20) if p["name"].startswith("tensor_action"))
        out["tensor_action_mf"] = {"kernel": "mf_cell_kernel + mf_row_kernel", "ms": pm["ms"],
                                   "achieved_gbs": pm["bytes"] / (pm["ms"] / 1e3) / 1e9,
                                   "frac_hbm": pm["bytes"] / (pm["ms"] / 1e3) / 1e9 / hbm,
                                   "bytes_per_launch": pm["bytes"], "speedup_vs_csf": csf["ms"] / pm["ms"]}
        hmf.close()

    if not args.no_next:
        # NEXT rows: the gradient coefficient (P0) and a quadrature space (I_3), same grid
        out["gradient_minsurf"] = next_row_extra(torch, P, dev, args.n, min(args.steps, 3), barrier, gradient_setup,
                                                 f"minimal_surface_p0_{args.n}x{args.n}", hbm, fp64_peak)
        out["quadrature_i3"] = next_row_extra(torch, P, dev, args.n, min(args.steps, 3), barrier, quadrature_setup,
                                              f"quadratic_reaction_i3_{args.n}x{args.n}", hbm, fp64_peak)
        out["superconductivity"] = supercond_extra(torch, P, dev, args.steps, barrier, hbm, fp64_peak, args.n)

    if not args.no_bratu:
        out["bratu_3d"] = bratu_extra(torch, P, dev, min(args.steps, 3), barrier, hbm, fp64_peak)

    if not args.no_batch:
        out["batched_adjoint"] = batched_adjoint_extra(torch, P, dev, args.batch_instances, args.batch_n, barrier)
        out["batched_p3"] = batched_p3_extra(torch, P, dev, args.p3_instances, barrier)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S = OracleSample(args.n, int(round(its["newton_iters"])), int(round(its["krylov_iters"])))
        threads = os.cpu_count() or 1
        s_all, per_all = S.step(threads)
        s_one, per_one = S.step(1)
        out["cpu_baseline"] = {"value": 1.0 / per_all, "unit": "solves/s", "cores": threads, "nproc": os.cpu_count(),
                               "kind": "oracle", "sample": S.desc, "sample_seconds": s_all,
                               "value_1_thread": 1.0 / per_one, "sample_seconds_1_thread": s_one}
    if rank == 0:
        print(json.dumps(out), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
