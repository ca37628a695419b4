"""Benchmark: time to a 1e-8 relative residual and skeleton-DOF·iterations/s.

Workload (the 2D generalized-Stokes scaling configuration at its largest
single-GPU size): unit square, 512x512 squares split into 524,288 triangles,
H(div)-HDG order k = 3 (6,283,264 skeleton unknowns), nu = 1, beta = 1,
gamma = 1e2 (eps^-1 = gamma nu), manufactured solution u = curl(sin^2(pi x)
sin^2(pi y)), p = sin(2 pi x) cos(2 pi y); hp-multigrid with lowest-order
(Crouzeix-Raviart) levels 32x32 ... 512x512 (5 levels; the 32x32 level solved exactly by one
dense FP64 GEMV with its precomputed inverse), variable V-cycle
(m_p = m_h = 1, doubling), FGMRES(15) inside the augmented-Lagrangian Uzawa
loop, stopping rules of Section 5 (inner relative 1e-8 / absolute 1e-10).

A step is one full solve (hdg_solve: Uzawa + FGMRES + hp-MG, all steps of the
hot path) from a zero initial guess on the condensed load resident in HBM.
Two forms are timed: FP64 throughout, and the mixed form (FP32
preconditioner inside FP64 FGMRES).  The headline value is the mixed form's
skeleton-DOF·iterations/s; both forms' time-to-tolerance are in the line.
Two further forms follow in "forms": the batched form (64 seeded loads on a
256x256 mesh solved together by hdg_solve_multi, against one load alone) and
the Oseen form (128x128, k = 2, Re = 1, 1e2, 1e3).

    python bench.py [--gpus 1] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the FP64 reference implementation of
the same method) on a bounded sample of the workload.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-8 rel. residual & skeleton-DOF·iters/s: FP64 plain vs mixed/batched"
UNIT = "skeleton-DOF·iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--N0", type=int, default=32,
                    help="coarsest CR level (exact dense FP64 solve); 32 keeps that solve one 290 MB GEMV")
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--gamma", type=float, default=1e2)
    ap.add_argument("--beta", type=float, default=1.0)
    ap.add_argument("--nu", type=float, default=1.0)
    ap.add_argument("--restart", type=int, default=15,
                    help="FGMRES restart length of the single-load solves (15 measured fastest at 512x512)")
    ap.add_argument("--restart-batched", type=int, default=8,
                    help="FGMRES restart length of the 64-load batched solve (8 measured fastest)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-forms", action="store_true",
                    help="skip the batched (64 loads) and Oseen forms")
    ap.add_argument("--profile-solve", action="store_true",
                    help="condense, then one warm-up and one timed mixed-precision solve only "
                         "(the command profiled for the kernel launch list)")
    ap.add_argument("--profile-precond-multi", action="store_true",
                    help="condense (--N, --k, --precision), then apply the batched preconditioner twice to 64 "
                         "seeded random columns (the command profiled for the batched smoother)")
    ap.add_argument("--profile-solve-multi", action="store_true",
                    help="condense --N (levels from 8x8), --k, --precision, then one warm-up and one batched solve of "
                         "64 seeded Fourier loads with FGMRES(--restart-batched) (the command profiled for the "
                         "batched solve's launch list)")
    ap.add_argument("--tetra-large", action="store_true",
                    help="add the 3D configuration at n = 48, k = 2 and 3 (23.6M and 39.4M unknowns, up to 229 GB) "
                         "to the 3D form")
    ap.add_argument("--profile-sweep3d", type=int, default=0, metavar="N",
                    help="3D: condense the N x N x N unit cube (Kuhn tetrahedra, levels from 2x2x2) at order --k "
                         "with the FP32 preconditioner, then run 4 order-k edge-patch sweeps (the command "
                         "profiled for the 3D sweep)")
    ap.add_argument("--precision", type=int, default=1,
                    help="preconditioner precision of --profile-solve / --profile-precond-multi "
                         "(hdg_precision value)")
    return ap.parse_args()


def workload(args):
    from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
    nl = 1
    while args.N0 * 2 ** (nl - 1) < args.N:
        nl += 1
    assert args.N0 * 2 ** (nl - 1) == args.N, "N must be N0 * 2^j"
    ms = unit_square_hierarchy(args.N0, nl)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, args.k,
                            curl_bubble_2d().forcing(args.nu, args.beta))
    return ms, fv


def solve_opts(hdg, restart):
    o = hdg.default_solve_opts()
    o.restart = restart
    return o


def config(args, n_dof, n_levels, l2="inputs larger than L2 (element and patch matrices several GB)"):
    return {"workload": f"2D generalized Stokes, unit square {args.N}x{args.N} (2N^2 triangles), "
                        f"H(div)-HDG k={args.k}, gamma={args.gamma:g}, alpha(beta)={args.beta:g}, "
                        f"nu={args.nu:g}, manufactured curl solution; hp-MG with CR levels "
                        f"{args.N0}x{args.N0}..{args.N}x{args.N} ({n_levels} levels), variable V-cycle "
                        f"m=1, FGMRES({args.restart}) in AL-Uzawa, stop rel 1e-8 / abs 1e-10",
            "N": args.N, "k": args.k, "skeleton_dofs": int(n_dof), "cells": 2 * args.N * args.N,
            "gamma": args.gamma, "beta": args.beta, "nu": args.nu,
            "restart": args.restart, "l2": l2}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        import statistics
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


_FINE = {}


def ctx_mesh_fine(args):
    return _FINE["mesh"]


def sweep_bytes(mesh, k, word, mat_word=None, packed_inverse=False, closed_form=False, al_split=False):
    """Bytes one order-k block-GS sweep (all colours) on `mesh` moves as the kernel reads them.

    Per vertex patch with nf interior facets (np = nf dpf unknowns) and nc cells:
    residual rows read 2 cells x dpf rows x n_loc columns per facet, the gathered
    cell unknowns nc x n_loc, the patch inverse np^2 (np (np+1)/2 when it is stored
    packed symmetric), the right-hand side np and the update np (read + write).
    In the closed form u_P = A_PP^-1 (g_P - A_PE u_E) the rows read only the dpf x dpf
    coupling block with the cell's facet opposite the patch vertex, the gather reads
    nc x dpf unknowns, and the update is written without being read.  The FP32 kernel's
    augmented-Lagrangian split (al_split) adds per patch the nc columns of Q (np_max rows each,
    as copied), one AL-free entry per (facet, cell) slot and the nc outside facets' FP64 flux
    weights.
    Vectors take `word` bytes per value, matrix entries `mat_word` (default `word`);
    16-bit matrices add one 4-byte scale per row read (2 x dpf per facet and np per
    patch inverse)."""
    import numpy as np
    dpf = 2 * (k + 1)
    nloc = 3 * dpf
    c = mesh.cells
    e = np.concatenate([c[:, [1, 2]], c[:, [0, 2]], c[:, [0, 1]]])
    e.sort(axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    interior = uniq[cnt == 2]
    nv = mesh.coords.shape[0]
    nf = np.bincount(interior.ravel(), minlength=nv)
    ncell = np.bincount(c.ravel(), minlength=nv)
    m = nf > 0
    npp = nf[m] * dpf
    mw = word if mat_word is None else mat_word
    inv = npp * (npp + 1) // 2 if packed_inverse else npp * npp
    cols, nx, nvec = (dpf, dpf, 2) if closed_form else (nloc, nloc, 3)
    mat = (nf[m] * 2 * dpf * cols + inv).sum() * mw
    vec = (ncell[m] * nx + nvec * npp).sum() * word
    scales = (nf[m] * 2 * dpf + npp).sum() * 4 if mw != word else 0
    split = ((ncell[m] * npp.max() + 2 * nf[m]).sum() * mw + ncell[m].sum() * 8) if al_split else 0
    return int(mat + vec + scales + split)


def patch_facet_counts(mesh):
    """Interior facets of every vertex patch (vertices with at least one) and cells of its star."""
    import numpy as np
    c = mesh.cells
    e = np.concatenate([c[:, [1, 2]], c[:, [0, 2]], c[:, [0, 1]]])
    e.sort(axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    interior = uniq[cnt == 2]
    nv = mesh.coords.shape[0]
    nf = np.bincount(interior.ravel(), minlength=nv)
    ncell = np.bincount(c.ravel(), minlength=nv)
    m = nf > 0
    return nf[m], ncell[m], int(interior.shape[0])


def survey_bytes(meshes, k, s_p=4, s_v=4, restart=30, m=1, growth=2):
    """Algorithmic bytes of the hot path by the per-unit model of the scope table
    (packed symmetric element matrices and patch inverses, each read once per use):
      A1  outer apply (FP64):        B_A + 2 N 8
      A2  one order-k sweep:         B_P + B_A' + 3 N s_v
      residual before Pi_k^0:        B_A' + 2 N s_v
      A4  MG_h, level l >= 1:        2 m(l) (B_P0 + B_A0 + 3 N_l s_v) + B_A0 + 4 N_l s_v,  m(J) = m,
                                     m(l-1) = growth m(l); level 0: the dense FP64 inverse, n0^2 8
      A6  CGS2 + flexible basis:     (4 restart/2 + 6) N 8
    B_A = n_cells n_loc (n_loc+1)/2 x 8, B_A' the same at s_p bytes, B_P = sum over patches of
    np (np+1)/2 x s_p; lowest-order quantities with dpf = 2."""
    dpf = 2 * (k + 1)
    nloc = 3 * dpf
    fine = meshes[-1]
    nf, _, n_int = patch_facet_counts(fine)
    N = n_int * dpf
    ncell = fine.cells.shape[0]
    npp = nf * dpf
    B_A = ncell * nloc * (nloc + 1) // 2 * 8
    B_Ap = ncell * nloc * (nloc + 1) // 2 * s_p
    B_P = int((npp * (npp + 1) // 2).sum()) * s_p
    out = {"A1_apply_fp64": B_A + 2 * N * 8,
           "A2_sweep": B_P + B_Ap + 3 * N * s_v,
           "residual_fp32": B_Ap + 2 * N * s_v,
           "A6_krylov": (4 * restart // 2 + 6) * N * 8}
    a4 = 0
    J = len(meshes) - 1
    ml = m
    for l in range(J, 0, -1):
        nf0, _, n0 = patch_facet_counts(meshes[l])
        N0 = 2 * n0
        B_P0 = int((2 * nf0 * (2 * nf0 + 1) // 2).sum()) * s_p
        B_A0 = meshes[l].cells.shape[0] * 21 * s_p
        a4 += 2 * ml * (B_P0 + B_A0 + 3 * N0 * s_v) + B_A0 + 4 * N0 * s_v
        ml *= growth
    _, _, nc0 = patch_facet_counts(meshes[0])
    a4 += (2 * nc0) ** 2 * 8
    out["A4_mg_h"] = a4
    out["B_it"] = (out["A1_apply_fp64"] + 2 * m * out["A2_sweep"] + out["residual_fp32"] + a4 + out["A6_krylov"])
    out["skeleton_dofs"] = N
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_baseline(args, seconds_budget=20.0):
    """The oracle (FP64, NumPy/SciPy) on a bounded sample of the workload: the same
    problem and method on a 32x32 triangulation (levels 8x8..32x32), timed for the
    solve phase only, like the GPU."""
    import numpy as np
    from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
    from oracle.topology import build_topology
    from oracle.hdg import HDG
    from oracle.mg import build_hpmg
    from oracle.krylov import uzawa
    N, N0 = 32, 8          # the sample keeps three lowest-order levels (8x8 .. 32x32)
    nl = 1
    while N0 * 2 ** (nl - 1) < N:
        nl += 1
    ms = unit_square_hierarchy(N0, nl)
    ts = [build_topology(m.coords, m.cells, m.vertex_colour) for m in ms]
    ps = [m.parent for m in ms]
    h = HDG(ts[-1], args.k, nu=args.nu, beta=args.beta, gamma=args.gamma)
    M = build_hpmg(ts, ps, args.k, args.nu, args.beta, args.gamma, hdg_k=h)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, args.k, curl_bubble_2d().forcing(args.nu, args.beta))
    F = h.load(fv)
    t0 = time.perf_counter()
    its = 0
    solves = 0
    while True:
        r = uzawa(M.A, h.flux_matrix(), h.area, h.eps_inv, F, M)
        its += sum(r.krylov_its)
        solves += 1
        if time.perf_counter() - t0 > seconds_budget or solves >= 3:
            break
    dt = time.perf_counter() - t0
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    return {"value": h.n_dof * its / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{solves} full solve(s) (Uzawa+FGMRES+hp-MG, FP64) of the same problem on a "
                      f"{N}x{N} triangulation, k={args.k}, {h.n_dof} skeleton DOFs; solve phase only; "
                      f"NumPy/SciPy threads as configured",
            "time_to_tol_s": dt / solves, "iters_per_solve": its / solves, "skeleton_dofs": h.n_dof}


def full_skeleton_dofs(N, k):
    """Skeleton unknowns of the N x N structured square: 3N^2 - 2N interior facets x 2(k+1)."""
    return (3 * N * N - 2 * N) * 2 * (k + 1)


def full_levels(args):
    nl = 1
    while args.N0 * 2 ** (nl - 1) < args.N:
        nl += 1
    return nl


def reference_arm(args):
    """--impl reference: the CPU oracle timed as the reference implementation."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
    from oracle.topology import build_topology
    from oracle.hdg import HDG
    from oracle.mg import build_hpmg
    from oracle.krylov import uzawa
    N, N0 = 32, 8          # the sample keeps three lowest-order levels (8x8 .. 32x32)
    nl = 1
    while N0 * 2 ** (nl - 1) < N:
        nl += 1
    ms = unit_square_hierarchy(N0, nl)
    ts = [build_topology(m.coords, m.cells, m.vertex_colour) for m in ms]
    ps = [m.parent for m in ms]
    h = HDG(ts[-1], args.k, nu=args.nu, beta=args.beta, gamma=args.gamma)
    M = build_hpmg(ts, ps, args.k, args.nu, args.beta, args.gamma, hdg_k=h)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, args.k, curl_bubble_2d().forcing(args.nu, args.beta))
    F = h.load(fv)
    D = h.flux_matrix()
    for _ in range(args.warmup):
        uzawa(M.A, D, h.area, h.eps_inv, F, M)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        r = uzawa(M.A, D, h.area, h.eps_inv, F, M)
        its += sum(r.krylov_its)
    dt = time.perf_counter() - t0
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    val = h.n_dof * its / dt
    # the config of what this arm times: the 32x32 sample of the workload
    sample_args = argparse.Namespace(**{**vars(args), "N": N, "N0": N0, "restart": 30})
    cfg = config(sample_args, h.n_dof, nl, l2="CPU run on the host cores (no GPU caches involved)")
    cfg["sample_of"] = f"{args.N}x{args.N} workload of the GPU arm ({full_skeleton_dofs(args.N, args.k)} skeleton DOFs)"
    sample = (f"{N}x{N} triangulation, {h.n_dof} skeleton DOFs, {nl} levels: a bounded CPU sample of the "
              f"{args.N}x{args.N} workload, timed over {args.steps} full solve(s)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def gpu_arm(args):
    import numpy as np
    import torch
    import paper_2303_06762_gb300 as hdg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # replicas only: every rank solves its own copy of the workload (no data-path collective)
    ms, fv = workload(args)
    _FINE["mesh"] = ms[-1]
    _FINE["meshes"] = ms
    ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=local)
    forcing = torch.tensor(fv, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = solve_opts(hdg, args.restart)
    results = {}
    sizes = None
    # (HDG_MIXED_BF16 is not timed here: at 512x512, k = 3 its FGMRES stalls before the
    # iteration limit; it is exercised by the parity tests on small meshes)
    for name, prec in (("fp64", hdg.HDG_FP64), ("mixed_fp32", hdg.HDG_MIXED_FP32),
                       ("mixed_fp16", hdg.HDG_MIXED_FP16)):
        prm = hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=args.gamma, precision=prec)
        torch.cuda.synchronize()
        t_setup = time.perf_counter()
        F = hdg.hdg_condense(ctx, prm, forcing)     # synchronises: condensation, inverses, coarse inverse
        t_setup = time.perf_counter() - t_setup
        sizes = ctx.sizes()
        u = torch.zeros(sizes.n_dof, dtype=torch.float64, device=dev)
        p = torch.zeros(sizes.n_cells, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            u.zero_(); p.zero_()
            hdg.hdg_solve(ctx, F, u, p, opts=opts)
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        l0 = hdg.hdg_kernel_launches()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        its = 0
        infos = []
        for _ in range(args.steps):
            u.zero_(); p.zero_()
            _, _, info = hdg.hdg_solve(ctx, F, u, p, opts=opts)
            its += info["krylov_its_total"]
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_total = ev0.elapsed_time(ev1)
        launches = hdg.hdg_kernel_launches() - l0
        clk = clocks.stop()
        if dist:
            t = torch.tensor([ms_total], device=dev)
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
            ms_total = float(t.item())
        dof_its = sizes.n_dof * its * world
        results[name] = {"time_to_tol_s": ms_total / 1e3 / args.steps,
                         "fgmres_iters_per_solve": its / args.steps,
                         "uzawa_steps": infos[-1]["uzawa_its"],
                         "krylov_its": infos[-1]["krylov_its"],
                         "dof_iters_per_s": dof_its / (ms_total / 1e3),
                         "ms_per_iter": ms_total / its if its else None,
                         "gpu_launches": launches, "clocks": clk, "F": F,
                         "setup_s": t_setup}
    head = results["mixed_fp32"]
    line = {"metric": METRIC, "value": head["dof_iters_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["time_to_tol_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (FGMRES, operator) / f32 (preconditioner)",
            "data": "synthetic", "config": config(args, sizes.n_dof, len(ms)),
            "forms": {n: {k: v for k, v in r.items() if k not in ("F", "clocks")}
                      for n, r in results.items()},
            "speedup_mixed_vs_fp64_time_to_tol": results["fp64"]["time_to_tol_s"] / head["time_to_tol_s"],
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
            "clocks_fp64": results["fp64"]["clocks"]}

    # ---------------------------------------------------------------- e2e: host buffers
    if not args.no_e2e:
        prm = hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=args.gamma,
                         precision=hdg.HDG_MIXED_FP32)
        F = hdg.hdg_condense(ctx, prm, forcing)
        F_host = F.cpu().pin_memory()
        u_host = torch.empty(sizes.n_dof, dtype=torch.float64).pin_memory()
        p_host = torch.empty(sizes.n_cells, dtype=torch.float64).pin_memory()
        Fd = torch.empty_like(F)
        u = torch.zeros_like(F)
        p = torch.zeros(sizes.n_cells, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        its = 0
        for _ in range(args.steps):
            Fd.copy_(F_host, non_blocking=True)
            u.zero_(); p.zero_()
            _, _, info = hdg.hdg_solve(ctx, Fd, u, p, opts=opts)
            its += info["krylov_its_total"]
            u_host.copy_(u, non_blocking=True)
            p_host.copy_(p, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        dt = ev0.elapsed_time(ev1) / 1e3
        line["e2e"] = {"value": sizes.n_dof * its * world / dt, "unit": UNIT,
                       "h2d_bytes_per_step": int(F.numel() * 8),
                       "d2h_bytes_per_step": int((u.numel() + p.numel()) * 8),
                       "time_to_tol_s": dt / args.steps}

    # ---------------------------------------------------------------- roofline of the dominant kernel
    line["roofline"] = roofline(args, ctx, hdg, torch, dev, stream, sizes)
    line["roofline_fp16_sweep"] = roofline(args, ctx, hdg, torch, dev, stream, sizes,
                                           precision=hdg.HDG_MIXED_FP16)
    ctx.close()
    fp64 = fp64_peak(hdg, torch, dev, stream)
    line["breakdown_mixed_iteration"] = breakdown(args, ms, hdg, torch, dev, stream, head["ms_per_iter"], fp64)
    comp = line["breakdown_mixed_iteration"]["components"]
    line["roofline"]["share_of_iteration"] = comp["order_k_sweeps"]["share_of_iteration"]
    line["roofline"]["largest_share"] = max((c for c in comp), key=lambda c: comp[c]["ms"])
    if not args.no_extra_forms:
        line["forms"]["batched_mixed_fp32"] = batched_form(args, hdg, torch, dev, stream, world)
        line["forms"]["oseen_mixed_fp32"] = oseen_form(args, hdg, torch, dev, stream)
        line["forms"]["coarsest_level_mixed_fp32"] = coarsest_form(args, hdg, torch, dev, stream)
        line["forms"]["variants_mixed_fp32"] = variants_form(args, ms, hdg, torch, dev, stream)
        line["forms"]["tetrahedra_3d"] = tetra_form(args, hdg, torch, dev, stream)

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        tdist.destroy_process_group()


def _timed(torch, stream, fn):
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    out = fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / 1e3, out


def batched_form(args, hdg, torch, dev, stream, world):
    """Many loads on one mesh: 2D 256x256 (131,072 triangles), k = 3, gamma = 1e2,
    beta = 1, nu = 1, 64 right-hand sides f_j = seeded Fourier sums plus gradient
    fields, solved together by hdg_solve_multi (mixed FP32 preconditioner), against
    one load solved alone by hdg_solve on the same operator."""
    from workloads import unit_square_hierarchy
    from workloads.manufactured import fourier_forcing_2d, lattice_points_2d
    # coarsest 8x8: with 64 columns the dense coarse solve is a GEMM of n0^2 x 64 FP64 products,
    # 4.6 GFLOP on a 32x32 coarsest level against 16 MFLOP on 8x8
    N, N0, k, nrhs = 256, 8, 3, 64
    nl = 1
    while N0 * 2 ** (nl - 1) < N:
        nl += 1
    ms = unit_square_hierarchy(N0, nl)
    fine = ms[-1]
    ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=dev.index or 0)
    prm = hdg.Params(k=k, nu=1.0, beta=1.0, gamma=1e2, precision=hdg.HDG_MIXED_FP32)
    hdg.hdg_condense(ctx, prm)
    X = torch.tensor(lattice_points_2d(fine.coords, fine.cells, k + 1), device=dev)
    shp = X.shape
    Xf = X.reshape(-1, 2)
    F = torch.stack([hdg.hdg_load(ctx, fourier_forcing_2d(j)(Xf, xp=torch).reshape(shp).contiguous())
                     for j in range(nrhs)])
    del X, Xf
    sizes = ctx.sizes()
    rb, nt, tile_ms = hdg.hdg_tune_batched(ctx, nrhs)  # the tile the autotuner keeps for this width
    om = solve_opts(hdg, args.restart_batched)
    hdg.hdg_solve_multi(ctx, F, opts=om)             # warm-up (graph capture, allocation)
    t, (U, P, infos) = _timed(torch, stream, lambda: hdg.hdg_solve_multi(ctx, F, opts=om))
    its = sum(i["krylov_its_total"] for i in infos)
    F0 = F[0].contiguous()
    o1 = solve_opts(hdg, args.restart)
    hdg.hdg_solve(ctx, F0, opts=o1)
    t1, (_, _, info1) = _timed(torch, stream, lambda: hdg.hdg_solve(ctx, F0, opts=o1))
    # the same loads with the order-k batched sweep on tensor cores (binary16 operands)
    hdg.hdg_condense(ctx, hdg.Params(k=k, nu=1.0, beta=1.0, gamma=1e2, precision=hdg.HDG_MIXED_FP16))
    _, nt_tc, ms_tc = hdg.hdg_tune_batched(ctx, nrhs)   # the tensor-core sweep's block size
    hdg.hdg_solve_multi(ctx, F, opts=om)
    th, (_, _, infos_h) = _timed(torch, stream, lambda: hdg.hdg_solve_multi(ctx, F, opts=om))
    its_h = sum(i["krylov_its_total"] for i in infos_h)
    ctx.close()
    uneven = uneven_meshes_form(hdg, torch, dev, stream, world, args.restart)
    return {"uneven_meshes": uneven,
            "workload": f"2D generalized Stokes {N}x{N} ({2 * N * N} triangles), k={k}, gamma=1e2, beta=1, nu=1, "
                        f"{nrhs} seeded Fourier+gradient loads, CR levels {N0}x{N0}..{N}x{N}, hdg_solve_multi",
            "nrhs": nrhs, "skeleton_dofs": int(sizes.n_dof), "time_to_tol_s": t,
            "fgmres_iters_total": its, "uzawa_steps_max": max(i["uzawa_its"] for i in infos),
            "dof_iters_per_s": sizes.n_dof * its * world / t,
            "single_load_time_to_tol_s": t1, "single_load_fgmres_iters": info1["krylov_its_total"],
            "single_load_dof_iters_per_s": sizes.n_dof * info1["krylov_its_total"] / t1,
            "throughput_ratio_vs_single": (sizes.n_dof * its / t) / (sizes.n_dof * info1["krylov_its_total"] / t1),
            "autotuned_tile": {"rows_per_thread": rb, "threads": nt, "colour_phase_ms": tile_ms},
            "tensor_core_fp16": {"time_to_tol_s": th, "fgmres_iters_total": its_h,
                                 "dof_iters_per_s": sizes.n_dof * its_h * world / th,
                                 "speedup_time_to_tol_vs_fp32": t / th,
                                 "autotuned_threads": nt_tc, "colour_phase_ms": ms_tc,
                                 "note": "HDG_MIXED_FP16: order-k batched sweep as mma.sync m16n8k16 with binary16 "
                                         "operands and FP32 accumulation"}}


def uneven_meshes_form(hdg, torch, dev, stream, world, restart=15):
    """Eight meshes N = 32, 64, ..., 256 (coarsest 2, 2, 3, 2, 5, 3, 7, 2), k = 3, one load each (the
    manufactured curl solution), mixed preconditioner: solved one after the other with hdg_solve, and
    concurrently with hdg_solve_batched (one host thread and stream per mesh), and as one solve of
    their disjoint union."""
    import numpy as np
    from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
    k = 3
    ctxs, Fs = [], []
    for N, N0 in ((32, 2), (64, 2), (96, 3), (128, 2), (160, 5), (192, 3), (224, 7), (256, 2)):
        nl = 1
        while N0 * 2 ** (nl - 1) < N:
            nl += 1
        ms = unit_square_hierarchy(N0, nl)
        fine = ms[-1]
        fv = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().forcing(1.0, 1.0))
        ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=dev.index or 0)
        Fs.append(hdg.hdg_condense(ctx, hdg.Params(k=k, nu=1.0, beta=1.0, gamma=1e2,
                                                     precision=hdg.HDG_MIXED_FP32), torch.tensor(fv, device=dev)))
        ctxs.append(ctx)
    dofs = [c.sizes().n_dof for c in ctxs]
    o = solve_opts(hdg, restart)
    for c, F in zip(ctxs, Fs):
        hdg.hdg_solve(c, F, opts=o)
    hdg.hdg_solve_batched(ctxs, Fs, opts=o)
    t_seq, its_seq = 0.0, []
    for c, F in zip(ctxs, Fs):
        t, (_, _, info) = _timed(torch, stream, lambda c=c, F=F: hdg.hdg_solve(c, F, opts=o))
        t_seq += t
        its_seq.append(info["krylov_its_total"])
    t0 = time.perf_counter()
    _, _, infos, stat = hdg.hdg_solve_batched(ctxs, Fs, opts=o)
    t_par = time.perf_counter() - t0
    its = [i["krylov_its_total"] for i in infos]
    work = sum(d * i for d, i in zip(dofs, its))
    for c in ctxs:
        c.close()
    # the same eight meshes as one disjoint union (every level of every mesh in one set of level
    # arrays: one context, one captured preconditioner graph, each launch covering all meshes);
    # the union needs equal depths, so every mesh gets 5 levels (coarsest N/16)
    from workloads.mesh2d import disjoint_union
    hs = [unit_square_hierarchy(N // 16, 5) for N in (32, 64, 96, 128, 160, 192, 224, 256)]
    un = disjoint_union(hs)
    fu = np.concatenate([forcing_at_lattice(h[-1].coords, h[-1].cells, k, curl_bubble_2d().forcing(1.0, 1.0))
                         for h in hs])
    cu = hdg.hdg_setup_mesh_hierarchy(un, device=dev.index or 0)
    Fu = hdg.hdg_condense(cu, hdg.Params(k=k, nu=1.0, beta=1.0, gamma=1e2, precision=hdg.HDG_MIXED_FP32),
                          torch.tensor(fu, device=dev))
    hdg.hdg_solve(cu, Fu, opts=o)
    t_un, (_, _, iu) = _timed(torch, stream, lambda: hdg.hdg_solve(cu, Fu, opts=o))
    nun = cu.sizes().n_dof
    cu.close()
    return {"meshes": [32, 64, 96, 128, 160, 192, 224, 256], "skeleton_dofs": dofs, "fgmres_iters": its,
            "sequential_s": t_seq, "concurrent_s": t_par,
            "dof_iters_per_s_sequential": sum(d * i for d, i in zip(dofs, its_seq)) * world / t_seq,
            "dof_iters_per_s_concurrent": work * world / t_par, "speedup": t_seq / t_par,
            "timing": "concurrent time is host wall clock around hdg_solve_batched, which synchronises",
            "union": {"time_to_tol_s": t_un, "fgmres_iters": iu["krylov_its_total"], "krylov_its": iu["krylov_its"],
                      "skeleton_dofs": int(nun), "levels": "5 per mesh (coarsest N/16)",
                      "speedup_vs_concurrent": t_par / t_un, "speedup_vs_sequential": t_seq / t_un,
                      "note": "one solve of the block-diagonal system of all eight meshes (shared Krylov "
                              "space and stopping rule), CUDA events"}}


def variants_form(args, ms, hdg, torch, dev, stream):
    """Solver variants.  On the headline workload (mixed form): PCG inner solves (Section 5) and
    the AL weight gamma = 1e4 (robustness in eps, reading r25 at scale).  The damped block-Jacobi
    smoother (eq. bjac, damping 1/2) and the additive hp-MG (Remark 3.4) need several times the
    iterations of block GS and grow with N (the oracle: Jacobi 67/96/114 and additive 230/382/>1000
    first-step iterations at N = 8/16/32 against GS 20/26/30), so they run on 128x128 (levels
    32x32..128x128) with FGMRES(30) and a bounded budget (at most 400 iterations per Uzawa step,
    8 Uzawa steps); `converged` says whether they met the stopping rule within it."""
    from workloads import curl_bubble_2d, forcing_at_lattice, unit_square_hierarchy
    out = {}

    def run(meshes, cases, restart, max_it=None, max_uzawa=None):
        fine = meshes[-1]
        fv = torch.tensor(forcing_at_lattice(fine.coords, fine.cells, args.k,
                                             curl_bubble_2d().forcing(args.nu, args.beta)), device=dev)
        ctx = hdg.hdg_setup_mesh_hierarchy(meshes, device=dev.index or 0)
        for name, extra, krylov, gamma in cases:
            prm = hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=gamma, precision=hdg.HDG_MIXED_FP32,
                             **extra)
            F = hdg.hdg_condense(ctx, prm, fv)
            o = solve_opts(hdg, restart)
            o.krylov = krylov
            if max_it:
                o.max_it, o.max_uzawa = max_it, max_uzawa
            t, (_, _, info) = _timed(torch, stream, lambda: hdg.hdg_solve(ctx, F, opts=o,
                                                                          raise_on_nonconvergence=False))
            out[name] = {"workload": f"{fine.N}x{fine.N}, k={args.k}, gamma={gamma:g}", "time_to_tol_s": t,
                         "krylov_its": info["krylov_its"][:info["uzawa_its"]],
                         "iterations": info["krylov_its_total"], "uzawa_steps": info["uzawa_its"],
                         "converged": info["converged"],
                         "res_floor_rel": info["res_floor"] / info["normF"], "div_l2": info["div_l2"]}
        ctx.close()

    run(ms, (("pcg", {}, 1, args.gamma), ("gamma_1e4", {}, 0, 1e4)), args.restart)
    run(unit_square_hierarchy(32, 3), (("block_jacobi", dict(smoother=1), 0, args.gamma),
                                       ("additive_hp_mg", dict(hp_additive=1), 0, args.gamma)),
        30, max_it=400, max_uzawa=8)
    return out


def coarsest_form(args, hdg, torch, dev, stream):
    """The headline workload (mixed form) with coarser or finer coarsest CR levels: fewer levels
    trade colour-phase launches of the small levels for a larger dense FP64 coarse inverse."""
    from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
    out = {}
    for N0 in (4, 8, 16, 32):
        if N0 == args.N0 or args.N % N0:
            continue
        nl = 1
        while N0 * 2 ** (nl - 1) < args.N:
            nl += 1
        ms = unit_square_hierarchy(N0, nl)
        fine = ms[-1]
        fv = forcing_at_lattice(fine.coords, fine.cells, args.k, curl_bubble_2d().forcing(args.nu, args.beta))
        ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=dev.index or 0)
        prm = hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=args.gamma, precision=hdg.HDG_MIXED_FP32)
        F = hdg.hdg_condense(ctx, prm, torch.tensor(fv, device=dev))
        o = solve_opts(hdg, args.restart)
        hdg.hdg_solve(ctx, F, opts=o)
        t, (_, _, info) = _timed(torch, stream, lambda: hdg.hdg_solve(ctx, F, opts=o))
        n = ctx.sizes().n_dof
        out[f"{N0}x{N0}"] = {"levels": nl, "time_to_tol_s": t, "fgmres_iters": info["krylov_its_total"],
                             "krylov_its": info["krylov_its"], "dof_iters_per_s": n * info["krylov_its_total"] / t,
                             "ms_per_iter": 1e3 * t / info["krylov_its_total"]}
        ctx.close()
    return out


def tetra_patch_sizes(cells):
    """Per edge patch of a tetrahedrisation (interior faces containing the edge): the number of
    patch faces and of star cells, for the byte models of the 3D sweep."""
    import numpy as np
    f = np.sort(np.concatenate([cells[:, [1, 2, 3]], cells[:, [0, 2, 3]], cells[:, [0, 1, 3]],
                                cells[:, [0, 1, 2]]]).astype(np.int64), axis=1)
    faces, cnt = np.unique(f, axis=0, return_counts=True)
    inner = faces[cnt == 2]
    e_of_faces = np.concatenate([inner[:, [0, 1]], inner[:, [0, 2]], inner[:, [1, 2]]])
    ce = np.sort(np.concatenate([cells[:, [a, b]] for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))]),
                 axis=1).astype(np.int64)
    nv = int(cells.max()) + 1
    key = lambda e: e[:, 0] * nv + e[:, 1]
    ek, star = np.unique(key(ce), return_counts=True)
    fk, nfac = np.unique(key(e_of_faces), return_counts=True)
    stars = star[np.searchsorted(ek, fk)]
    return nfac, stars, len(inner)


def tetra_sweep_bytes(cells, k, word=4):
    """Bytes of one order-k block GS sweep over edge patches in 3D (all colours), two models:
    the scope table's per-unit model B_P (packed symmetric patch inverses) + B_A' (packed
    symmetric element matrices) + 3 N s_v, and the kernel's own accesses (full transposed
    patch inverses, both cells' row blocks of every patch face, the star cells' unknowns, g, u)."""
    import numpy as np
    nf = (k + 1) * (k + 2) // 2
    dpf = 3 * nf
    nloc = 4 * dpf
    nfac, stars, n_int = tetra_patch_sizes(cells)
    npch = nfac * dpf
    N = n_int * dpf
    model = word * (np.sum(npch * (npch + 1) // 2) + cells.shape[0] * nloc * (nloc + 1) // 2 + 3 * N)
    kernel = word * (np.sum(npch * npch) + np.sum(2 * nfac * nloc * dpf) + np.sum(stars * nloc) + 3 * np.sum(npch))
    return int(model), int(kernel)


def tetra_form(args, hdg, torch, dev, stream):
    """The 3D configuration (Section 5.1.2 workloads): the unit cube in n^3 cubes of 6 Kuhn
    tetrahedra, a red-refined hierarchy 2x2x2 -> ... -> n, beta = 1, nu = 1, gamma = 1e2, the
    manufactured curl solution, edge-patch block GS with two smoothing steps (m_p = m_h = 2, the
    paper's 3D setting: half the iterations of m = 1 and 20% less time, measured); FP64 and the
    FP32 preconditioner, FGMRES(30) in AL-Uzawa with the default stopping rule; the mixed
    order-k sweep against its rooflines."""
    from workloads.mesh3d import unit_cube_hierarchy
    from workloads.manufactured import curl_bubble_3d, forcing_at_lattice
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    out = {}
    cases = [(2, 4, 2, ("fp64", "mixed_fp32")), (2, 4, 3, ("fp64", "mixed_fp32")), (2, 5, 2, ("mixed_fp32",)),
             (2, 5, 3, ("mixed_fp32",))]
    if getattr(args, "tetra_large", False):
        # n = 48 (hierarchy 3 -> 6 -> 12 -> 24 -> 48): about 162 GB (k = 2) and 229 GB (k = 3) on the device
        cases += [(3, 5, 2, ("mixed_fp32",)), (3, 5, 3, ("mixed_fp32",))]
    for n0, nl, k, forms in cases:
        ms = unit_cube_hierarchy(n0, nl)
        fine = ms[-1]
        n = n0 * 2 ** (nl - 1)
        fv = torch.tensor(forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_3d().forcing(1.0, 1.0)),
                          device=dev)
        ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=dev.index or 0)
        rec = {"n": n, "k": k, "tetrahedra": int(fine.n_cells), "levels": nl}
        for name in forms:
            prec = hdg.HDG_FP64 if name == "fp64" else hdg.HDG_MIXED_FP32
            prm = hdg.Params(k=k, nu=1.0, beta=1.0, gamma=1e2, precision=prec, m_p=2, m_h=2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F = hdg.hdg_condense(ctx, prm, fv)
            torch.cuda.synchronize()
            setup = time.perf_counter() - t0
            o = solve_opts(hdg, 30 if n < 48 else 15)   # n = 48: FGMRES(15) keeps the basis at 10 GB
            hdg.hdg_solve(ctx, F, opts=o)
            t, (u, p, info) = _timed(torch, stream, lambda: hdg.hdg_solve(ctx, F, opts=o))
            nd = ctx.sizes().n_dof
            rec["skeleton_dofs"] = int(nd)
            rec[name] = {"time_to_tol_s": t, "fgmres_iters": info["krylov_its_total"],
                         "krylov_its": info["krylov_its"], "uzawa_steps": info["uzawa_its"],
                         "dof_iters_per_s": nd * info["krylov_its_total"] / t,
                         "ms_per_iter": 1e3 * t / max(info["krylov_its_total"], 1), "setup_s": setup,
                         "div_l2": info["div_l2"]}
        # the mixed form's order-k sweep (all colours) against both byte models
        r = torch.randn(ctx.sizes().n_dof, dtype=torch.float64, device=dev)
        z = torch.zeros_like(r)
        t_sw = _event_ms(torch, stream, lambda: hdg.hdg_smooth(ctx, -1, r, z, 4, False), 3) / 4
        bm, bk = tetra_sweep_bytes(fine.cells, k)
        rec["sweep_mixed"] = {"kernel": "gs3_kernel<float,%d> (edge patches, %d colour launches)"
                              % (3 * (k + 1) * (k + 2) // 2, int(ctx.sizes().n_colours_level[nl - 1])),
                              "ms": t_sw, "model_bytes": bm, "kernel_bytes": bk,
                              "frac_by_model": bm / (t_sw / 1e3) / 1e9 / peak,
                              "frac_by_kernel_bytes": bk / (t_sw / 1e3) / 1e9 / peak,
                              "peak_gbs": peak, "note": "includes the FP64<->FP32 conversions of g and u"}
        out[f"n{n}_k{k}"] = rec
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    return out


def oseen_form(args, hdg, torch, dev, stream):
    """Oseen: 128x128 (32,768 triangles), k = 2, gamma = 1e2, beta = 0, upwind
    convection by b = curl(sin^2(pi x) sin^2(pi y)) scaled to max|b| = 1, nu = 1/Re."""
    from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice
    from workloads.manufactured import convecting_stream_2d, curl_lattice_2d
    N, N0, k = 128, 8, 2
    nl = 1
    while N0 * 2 ** (nl - 1) < N:
        nl += 1
    ms = unit_square_hierarchy(N0, nl)
    fine = ms[-1]
    psi, b = convecting_stream_2d(1.0)
    conv = torch.tensor(curl_lattice_2d(fine.coords, fine.cells, k + 1, psi), device=dev)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=dev.index or 0)
    out = {"workload": f"2D Oseen {N}x{N} ({2 * N * N} triangles), k={k}, gamma=1e2, beta=0, "
                       f"b=curl(sin^2 pi x sin^2 pi y) with max|b|=1, nu=1/Re, CR levels {N0}x{N0}..{N}x{N}"}
    for Re in (1.0, 1e2, 1e3):
        nu = 1.0 / Re
        fv = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().forcing(nu, 0.0, conv=b))
        prm = hdg.Params(k=k, nu=nu, beta=0.0, gamma=1e2, precision=hdg.HDG_MIXED_FP32, conv=conv)
        F = hdg.hdg_condense(ctx, prm, torch.tensor(fv, device=dev))
        o = solve_opts(hdg, 50)          # the Oseen configuration's FGMRES(50)
        hdg.hdg_solve(ctx, F, opts=o, raise_on_nonconvergence=False)
        t, (_, _, info) = _timed(torch, stream, lambda: hdg.hdg_solve(ctx, F, opts=o, raise_on_nonconvergence=False))
        n = ctx.sizes().n_dof
        out[f"Re={Re:g}"] = {"time_to_tol_s": t, "fgmres_iters": info["krylov_its_total"],
                             "uzawa_steps": info["uzawa_its"], "dp_rel": info["dp_rel"],
                             "dof_iters_per_s": n * info["krylov_its_total"] / t}
    out["skeleton_dofs"] = int(ctx.sizes().n_dof)
    ctx.close()
    return out


def _event_ms(torch, stream, fn, reps):
    """Mean milliseconds of fn() over reps calls, CUDA events on `stream`, after one warm-up."""
    fn()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


def fp64_peak(hdg, torch, dev, stream):
    """FP64 FMA rate of this GPU (TFLOP/s) from the library's probe kernel, best of 3."""
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    best = 0.0
    for _ in range(3):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        flops = hdg.hdg_fp64_fma_probe(out, 8, 1 << 15)
        ev1.record(stream)
        torch.cuda.synchronize()
        best = max(best, flops / (ev0.elapsed_time(ev1) / 1e3) / 1e12)
    return best


def breakdown(args, ms, hdg, torch, dev, stream, ms_per_iter, fp64_tflops):
    """One FGMRES iteration of the mixed form taken apart with CUDA events: the preconditioner
    application, its two order-k sweeps and its lowest-order V-cycle MG_h, the FP64 outer apply,
    and the rest (Gram-Schmidt, Givens, the per-iteration residual read); each against the
    scope table's algorithmic bytes (survey_bytes) and the measured HBM peak, the FP64 apply
    also against the FP64 FMA rate."""
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms, device=dev.index or 0)
    prm = hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=args.gamma, precision=hdg.HDG_MIXED_FP32)
    hdg.hdg_condense(ctx, prm, None)
    n = ctx.sizes().n_dof
    gen = torch.Generator(device=dev).manual_seed(3)
    r = torch.randn(n, dtype=torch.float64, device=dev, generator=gen)
    z = torch.empty_like(r)
    n0 = int(ctx.sizes().n_dof_level[len(ms) - 1])
    g0 = torch.randn(n0, dtype=torch.float64, device=dev, generator=gen)
    u0 = torch.empty_like(g0)
    t_pc = _event_ms(torch, stream, lambda: hdg.hdg_precond_apply(ctx, r, z), 10)
    # MG_h is several hundred small launches: capture one application in a CUDA graph and time
    # its replays, as the preconditioner's own graph runs it inside hdg_precond_apply
    hdg.hdg_mg_h(ctx, g0, u0)
    torch.cuda.synchronize()
    side = torch.cuda.Stream(device=dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        hdg.hdg_mg_h(ctx, g0, u0)
    t_mgh = _event_ms(torch, stream, graph.replay, 10)
    t_ap = _event_ms(torch, stream, lambda: hdg.hdg_apply(ctx, r, z), 10)
    u = torch.zeros_like(r)
    t_sw = _event_ms(torch, stream, lambda: hdg.hdg_smooth(ctx, -1, r, u, 4, False), 3) / 4
    ctx.close()
    b = survey_bytes(ms, args.k)
    dpf = 2 * (args.k + 1)
    nloc = 3 * dpf
    ncell = ms[-1].cells.shape[0]
    comp = {
        "order_k_sweeps": {"ms": 2 * t_sw, "bytes": 2 * b["A2_sweep"],
                           "kernel": "gs_tma_kernel<8> (x 2 sweeps x 3 colours)"},
        "mg_h": {"ms": t_mgh, "bytes": b["A4_mg_h"],
                 "kernel": "lowest-order V-cycle: gs0t_kernel/gs0_kernel<float,16>, transfers, coarse GEMV"},
        "apply_fp64": {"ms": t_ap, "bytes": b["A1_apply_fp64"], "kernel": "apply_kernel<double,8>",
                       "fp64_tflops": 2.0 * ncell * nloc * nloc / (t_ap / 1e3) / 1e12},
    }
    rest = ms_per_iter - t_pc - t_ap
    comp["krylov_and_rest"] = {"ms": rest, "bytes": b["A6_krylov"],
                               "kernel": "dots_kernel, update_dots_kernel, givens, scale (CGS2)"}
    comp["precond_other"] = {"ms": t_pc - 2 * t_sw - t_mgh, "bytes": b["residual_fp32"],
                             "kernel": "FP32 residual apply, Pi_k^0 transfers, conversions"}
    for c in comp.values():
        c["share_of_iteration"] = c["ms"] / ms_per_iter
        c["achieved_gbs"] = c["bytes"] / (c["ms"] / 1e3) / 1e9 if c["ms"] > 0 else None
        c["frac_of_hbm"] = c["achieved_gbs"] / peak if c["achieved_gbs"] else None
    comp["apply_fp64"]["frac_of_fp64"] = comp["apply_fp64"]["fp64_tflops"] / fp64_tflops if fp64_tflops else None
    return {"ms_per_iter": ms_per_iter, "precond_ms": t_pc, "components": comp,
            "fp64_fma_tflops_measured": fp64_tflops,
            "survey_bytes_per_iteration": b["B_it"],
            "iteration_frac_of_hbm": b["B_it"] / (ms_per_iter / 1e3) / 1e9 / peak,
            "ideal_ms_per_iter": b["B_it"] / (peak * 1e9) * 1e3}


def roofline(args, ctx, hdg, torch, dev, stream, sizes, precision=None):
    """Order-k block Gauss-Seidel sweep in FP32 (the mixed form's dominant kernel),
    timed with CUDA events on the launching stream over 20 sweeps; with
    precision = HDG_MIXED_FP16 the same sweep on the binary16 matrix copies.

    Algorithmic bytes per sweep (one launch per colour, 3 colours): every cell's
    condensed matrix is read for the two facets at the patch vertex in each of the
    three colour phases (2 x n_loc^2 x 4 B per cell), every patch inverse once
    (np^2 x 4 B), and the right-hand side, solution gather and update
    (about 2 reads + 1 write of the unknowns of each patch, 4 B each)."""
    peaks = measured_peaks()
    k = args.k
    nloc = 6 * (k + 1)
    dpf = 2 * (k + 1)
    half = precision == hdg.HDG_MIXED_FP16
    prm = hdg.Params(k=k, nu=args.nu, beta=args.beta, gamma=args.gamma,
                     precision=hdg.HDG_MIXED_FP32 if precision is None else precision)
    hdg.hdg_condense(ctx, prm, None)
    g = torch.randn(sizes.n_dof, dtype=torch.float64, device=dev)
    u = torch.zeros_like(g)
    n_sweeps = 20
    hdg.hdg_smooth(ctx, -1, g, u, 3, False)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    hdg.hdg_smooth(ctx, -1, g, u, n_sweeps, False)
    ev1.record(stream)
    torch.cuda.synchronize()
    # hdg_smooth converts g, u to FP32 and back once per call: subtract that traffic's time
    # by timing a zero-sweep call
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    hdg.hdg_smooth(ctx, -1, g, u, 0, False)
    ev3.record(stream)
    torch.cuda.synchronize()
    t_sweep = (ev0.elapsed_time(ev1) - ev2.elapsed_time(ev3)) / 1e3 / n_sweeps
    # algorithmic bytes by the scope table's per-unit model (packed symmetric element matrices
    # and patch inverses read once per sweep), and by the kernel's own full-storage access count
    alg = survey_bytes(_FINE["meshes"], k, s_p=2 if half else 4)["A2_sweep"]
    alg_kernel = sweep_bytes(ctx_mesh_fine(args), k, 4, 2 if half else 4, packed_inverse=not half,
                             closed_form=not half, al_split=not half)
    achieved = alg / t_sweep / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    # DRAM bytes of one sweep from an ncu capture of the same kernel on the 128x128, k = 3 case
    # (TMA_SWEEP_TRAFFIC_128).  Traffic grows with the number of patches like the algorithmic
    # bytes, so the full-size figure is that ratio times the full-size algorithmic bytes
    # (k = 3 only; other k were not captured).
    traffic = alg_kernel * (TMA_SWEEP_TRAFFIC_128 / TMA_SWEEP_KERNEL_BYTES_128) \
        if k == 3 and not half and TMA_SWEEP_TRAFFIC_128 else None
    kname = "gs_kernel<float, 8, __half> (order-k block GS sweep on binary16 copies" if half else \
        "gs_tma_kernel<8> (order-k block GS sweep, matrices staged by cp.async.bulk"
    rs = read_stream_gbs(torch, dev, stream)
    return {"kernel": kname + ", 3 colour launches)",
            "read_stream_gbs": rs, "frac_of_read_stream": achieved / rs,
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_note": ("per sweep (3 colour launches), like achieved: the ncu DRAM bytes of one sweep at 128x128 "
                             "scaled by the kernel bytes to 512x512 (same kernel, cold caches)") if traffic else None,
            "traffic_over_algorithmic": traffic / alg if traffic else None,
            "algorithmic_bytes_per_sweep": alg,
            "bytes_model": "scope table per-unit model: B_P + B_A' + 3 N s_v (packed symmetric)",
            "kernel_access_bytes_per_sweep": alg_kernel,
            "frac_by_kernel_access_bytes": alg_kernel / t_sweep / 1e9 / peak,
            "sweep_ms": t_sweep * 1e3,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the three colour launches of one
# order-k sweep of gs_tma_kernel<8, 1> (closed form with the AL split, packed symmetric patch
# inverses) from an ncu capture on the 128x128, k = 3 case (profiles/ncu_gs_tma_closed_form_128_k3.md),
# and that sweep's bytes as the kernel reads them (sweep_bytes, packed inverse, closed form, split):
# (54,397,696 + 115,712) + (54,395,648 + 113,152) + (54,387,200 + 128,768) B against 156,064,048 B.
TMA_SWEEP_TRAFFIC_128 = 163538176
TMA_SWEEP_KERNEL_BYTES_128 = 156064048


def read_stream_gbs(torch, dev, stream):
    """Read-only streaming rate of this GPU: a full reduction over 2 GiB (larger than L2),
    the ceiling for a kernel that, like the sweep, reads matrices and writes little."""
    x = torch.ones(1 << 29, dtype=torch.float32, device=dev)
    x.sum()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(10):
        x.sum()
    ev1.record(stream)
    torch.cuda.synchronize()
    gbs = x.numel() * 4 * 10 / (ev0.elapsed_time(ev1) / 1e3) / 1e9
    del x
    return gbs


def profile_solve(args):
    import torch
    import paper_2303_06762_gb300 as hdg
    ms, fv = workload(args)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    prm = hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=args.gamma, precision=args.precision)
    F = hdg.hdg_condense(ctx, prm, torch.tensor(fv, device="cuda:0"))
    for _ in range(max(args.warmup, 0) + 1):
        u, p, info = hdg.hdg_solve(ctx, F, opts=solve_opts(hdg, args.restart))
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": True, "N": args.N, "k": args.k, "launches": hdg.hdg_kernel_launches(),
                      "info": info}))
    ctx.close()


def profile_precond_multi(args):
    import torch
    import paper_2303_06762_gb300 as hdg
    ms, _ = workload(args)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=args.k, nu=args.nu, beta=args.beta, gamma=args.gamma,
                                     precision=args.precision))
    gen = torch.Generator(device="cuda:0").manual_seed(1)
    X = torch.randn((64, ctx.sizes().n_dof), dtype=torch.float64, device="cuda:0", generator=gen)
    for _ in range(2):
        Z = hdg.hdg_precond_apply_multi(ctx, X)
    torch.cuda.synchronize()
    print(json.dumps({"profile_precond_multi": True, "N": args.N, "k": args.k, "precision": args.precision,
                      "max_abs": float(Z.abs().max())}))
    ctx.close()


def profile_solve_multi(args):
    import torch
    import paper_2303_06762_gb300 as hdg
    from workloads import unit_square_hierarchy
    from workloads.manufactured import fourier_forcing_2d, lattice_points_2d
    nl = 1
    while 8 * 2 ** (nl - 1) < args.N:
        nl += 1
    ms = unit_square_hierarchy(8, nl)
    fine = ms[-1]
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=args.k, nu=1.0, beta=1.0, gamma=1e2, precision=args.precision))
    X = torch.tensor(lattice_points_2d(fine.coords, fine.cells, args.k + 1), device="cuda:0")
    shp = X.shape
    F = torch.stack([hdg.hdg_load(ctx, fourier_forcing_2d(j)(X.reshape(-1, 2), xp=torch).reshape(shp).contiguous())
                     for j in range(64)])
    o = solve_opts(hdg, args.restart_batched)
    for _ in range(2):
        U, P, infos = hdg.hdg_solve_multi(ctx, F, opts=o)
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve_multi": True, "N": args.N, "k": args.k, "precision": args.precision,
                      "iterations": sum(i["krylov_its_total"] for i in infos),
                      "launches": hdg.hdg_kernel_launches()}))
    ctx.close()


def profile_sweep3d(args):
    import torch
    import paper_2303_06762_gb300 as hdg
    from workloads.mesh3d import unit_cube_hierarchy
    nl = 1
    while 2 ** nl < args.profile_sweep3d:
        nl += 1
    ms = unit_cube_hierarchy(2, nl)
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    hdg.hdg_condense(ctx, hdg.Params(k=args.k, nu=1.0, beta=1.0, gamma=1e2, precision=hdg.HDG_MIXED_FP32))
    gen = torch.Generator(device="cuda:0").manual_seed(1)
    g = torch.randn(ctx.sizes().n_dof, dtype=torch.float64, device="cuda:0", generator=gen)
    u = torch.zeros_like(g)
    hdg.hdg_smooth(ctx, -1, g, u, 4, False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_sweep3d": True, "n": 2 ** nl, "k": args.k, "max_abs": float(u.abs().max())}))
    ctx.close()


def main():
    args = parse()
    if args.profile_sweep3d:
        profile_sweep3d(args)
        return
    if args.profile_solve_multi:
        profile_solve_multi(args)
        return
    if args.profile_solve:
        profile_solve(args)
        return
    if args.profile_precond_multi:
        profile_precond_multi(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    gpu_arm(args)


if __name__ == "__main__":
    main()
