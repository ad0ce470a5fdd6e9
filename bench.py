"""Benchmark: full multigrid-preconditioned CG solve to relative residual 1e-6.

One step = one ocg_pcg_solve (Alg. 1 with one FAS-style V-cycle per iteration) of the
two-level octree workload: 64^3 root grid, cells whose centre lies within 0.25 of the
cube centre refined once (382,936 leaves), beta = 1, Dirichlet walls, manufactured
p = exp(x) sin(2 pi y) cos(2 pi z); FP32 cycle inside FP64 PCG ("mixed"), with the plain
FP32 solve reported beside it.  Inputs are resident in HBM before the timed region; L2
is flushed (256 MB write) before every timed step.  Under torchrun every rank solves
its own replica (the path does not shard below one octree): weak scaling, no
collective in the data path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve Mcells/s at rel-res 1e-6 (mixed/batched vs plain FP32), % HBM roof"
UNIT = "Mcells/s"
WORKLOAD = ("octree 64^3 root, ball r=0.25 at the centre refined once (382,936 leaves, "
            "effective 128^3), beta=1, Dirichlet walls, p=exp(x)sin(2pi y)cos(2pi z)")
# algorithmic bytes per cell of one red-black colour sweep: 16 B coefficients (c, c_x-,
# c_y-, c_z- in FP32) + 4 B u read + 2 B u write (half the cells) + 2 B b (half)
SWEEP_BYTES_PER_CELL = 24.0
NOMINAL_HBM_GBS = 7700.0   # B300 HBM3e nominal bandwidth, for a second fraction beside the measured one


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("kernels.cuh", "octet.cuh", "ocg_api.cu"):
        with open(os.path.join(ROOT, "paper_2604_18886_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(name, cells):
    """DRAM bytes (read + write) of one launch of a probed kernel on `cells` cells, from the
    committed ncu summary profiles/<name>.txt (per-cell bytes of the captured launch) when
    that summary was taken on the current kernel sources; None otherwise."""
    p = os.path.join(ROOT, "profiles", name + ".txt")
    try:
        kv = {}
        for line in open(p):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_hash") == _kernel_hash():
            return round(float(kv["dram_bytes_per_cell"]) * cells)
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi samples (every 20 ms) of SM clock, power and throttle reasons; started
    before the timed region, which is bracketed by line marks."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def _rows(self):
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and line.endswith("\n"):
                    rows.append(parts)
        except Exception:
            pass
        return rows

    def wait_first(self, timeout=15.0):
        t_end = time.time() + timeout
        while self.p is not None and time.time() < t_end and not self._rows():
            time.sleep(0.05)

    def mark(self):
        return len(self._rows())

    def stop(self, lo, hi):
        if self.p is None:
            return None
        time.sleep(0.05)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        rows = self._rows()
        os.unlink(self.f.name)
        inside = rows[lo:hi + 1]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "no nvidia-smi sample fell inside the timed region"}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in inside if num(r[1]) is not None]
        mx = [num(r[2]) for r in inside if num(r[2]) is not None]
        pw = [num(r[3]) for r in inside if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w": statistics.median(pw) if pw else None, "reasons": reasons, "samples": len(inside)}


def _setup(dev, sweep="auto"):
    import numpy as np
    import torch
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S
    p = P.two_level_ball(64)
    tree = S.Octree(p.desc)
    faces = tree.faces()
    beta = P.face_beta(p, faces)
    hier = S.Hierarchy(tree, torch.from_numpy(beta).to(dev), p.bc, S.mg_params(coef="f32", sweep=sweep))
    b = P.rhs(p, tree.leaves(), faces, beta)
    return p, tree, hier, torch.from_numpy(b).to(dev), np


def max_over_ranks(v, dev):
    """Largest value of v over the ranks of the default process group (v itself when
    there is none): the timed region is as long as its slowest replica."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, steps, world, total_ms):
    """Whole-job throughput in millions of units per second: every rank solves its own
    replica, total_ms is the slowest rank's timed region."""
    return world * units_per_rank * steps / (total_ms / 1e3) / 1e6


def _hier_bf16(p, tree, dev):
    import torch
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S
    beta = P.face_beta(p, tree.faces())
    return S.Hierarchy(tree, torch.from_numpy(beta).to(dev), p.bc, S.mg_params(coef="f32", bf16_coarse=True))


HYBRID_MIN_CELLS = 1 << 20


def _w_cycle(g, beta, p, b, dev, stream, flush, steps, bf16=False, mu_min_cells=0):
    """The same solve preconditioned by W-cycles (mu = 2; the paper's choice for cut-cell
    problems) instead of V-cycles: iterations and Mcells/s.  mu_min_cells > 0: mu = 2 only
    into levels with at least that many cells (V below)."""
    import torch
    from paper_2604_18886_b300 import solver as S
    hw = S.Hierarchy(g, beta, p.bc, S.mg_params(mu=2, coef="f32", bf16_coarse=bf16, mu_min_cells=mu_min_cells))
    x = torch.empty_like(b)
    hw.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
    t, its = [], set()
    for s_ in range(steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = hw.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
        e1.record(stream)
        e1.synchronize()
        t.append(e0.elapsed_time(e1))
        its.add(st.iterations)
    ms = statistics.mean(t)
    del hw
    return {"value": round(g.n_leaves / (ms / 1e3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms, 3),
            "iterations": sorted(its), "true_rel_res": st.true_rel_res,
            "cycle": ("W (mu=2) into levels of >= %d cells, V below, nu=2/2" % mu_min_cells) if mu_min_cells
            else "W (mu=2), nu=2/2"}


def _cut_cell(dev, stream, flush, args):
    """The cut-cell projection workload: 64^3 root, two levels of refinement within 0.05
    of a solid sphere and box, fluid-fraction beta, Neumann walls, divergence rhs; mixed
    solve with BF16 coarse coefficients to 1e-6."""
    import torch
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S
    p = P.cut_cell(64, 2)
    g = S.Octree(p.desc)
    f = g.faces()
    beta = P.face_beta(p, f)
    h = S.Hierarchy(g, torch.from_numpy(beta).to(dev), p.bc, S.mg_params(coef="f32", bf16_coarse=True))
    b = torch.from_numpy(P.rhs(p, g.leaves(), f, beta)).to(dev)
    x = torch.empty_like(b)
    for _ in range(args.warmup):
        h.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
    steps = max(3, min(args.steps, 20))
    t, its = [], set()
    for s_ in range(steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = h.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
        e1.record(stream)
        e1.synchronize()
        t.append(e0.elapsed_time(e1))
        its.add(st.iterations)
        assert st.converged
    ms = statistics.mean(t)
    wc = _w_cycle(g, beta, p, b, dev, stream, flush, steps, bf16=True)
    wh = _w_cycle(g, beta, p, b, dev, stream, flush, steps, bf16=True, mu_min_cells=HYBRID_MIN_CELLS)
    # ablation (Sec. 3.3): geometric multigrid, coarse cells rediscretised from the solids
    hg = S.Hierarchy(g, torch.from_numpy(beta).to(dev), p.bc, S.mg_params(coef="f32", coarsening="geometric"))
    hg.solve(b, x, tol=1e-6, precision="mixed", stream=stream, max_iter=400)
    flush.fill_(0.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, sg = hg.solve(b, x, tol=1e-6, precision="mixed", stream=stream, max_iter=400)
    e1.record(stream)
    e1.synchronize()
    msg = e0.elapsed_time(e1)
    gmg = {"value": round(g.n_leaves / (msg / 1e3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(msg, 3),
           "iterations": sg.iterations, "converged": bool(sg.converged),
           "what": "geometric coarsening (Sec. 3.3 ablation), V-cycle, mixed, FP32 coefficients"}
    del hg
    return {"w_cycle": wc, "w_v_hybrid": wh, "geometric_coarsening": gmg,
            "workload": "cut-cell projection: 64^3 root, sphere r=0.2 and box, band 0.05, 2 levels "
                        "(%d leaves), fluid-fraction beta, Neumann, divergence rhs" % g.n_leaves,
            "precision": "mixed, BF16 coarse coefficients", "value": round(g.n_leaves / (ms / 1e3) / 1e6, 3),
            "unit": UNIT, "ms_per_step": round(ms, 4), "steps": steps, "iterations": sorted(its),
            "true_rel_res": st.true_rel_res}


LARGE_WORKLOAD = ("large differentiable solve: 128^3 root refined 3 times within 0.02 (+ cell reach) of the "
                  "zero set of 8 seeded plane sine waves (effective 1024^3), fluid-fraction beta, Neumann, "
                  "divergence rhs")


def _tank(dev, stream, flush, args):
    """The static tank (Sec. 4.4): liquid in [0,1]^3, solid bottom and sides, open top, a
    cut-cell sphere or star obstacle; the 64^3 root with two levels near the obstacle is
    the paper's 64~256 grid.  Mixed solves to 1e-6 with W-cycles (the paper's choice here)
    and V-cycles: iterations, mean residual reduction per iteration, time, the largest
    deviation from the exact discrete pressure y - 1 and the divergence of the projected
    velocity relative to the initial one (volume-weighted RMS)."""
    import math
    import numpy as np
    import torch
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S
    out = {}
    cases = [(o, n0, True) for o in ("sphere", "star") for n0 in (64, 128)] + \
        [(o, 64, False) for o in ("sphere", "star")]
    for obstacle, n0, inactive in cases:
        if True:
            p = P.tank(obstacle, n0, inactive)
            g = S.Octree(p.desc)
            f = g.faces()
            beta = P.face_beta(p, f)
            lv = g.leaves()
            b = torch.from_numpy(P.rhs(p, lv, f, beta)).to(dev)
            hc, xc, yc, zc = P.leaf_centres(n0, lv)
            ref = torch.from_numpy(yc - 1.0).to(dev)
            V = torch.from_numpy(hc ** 3).to(dev)
            row = {"leaves": g.n_leaves}
            for mu in (2, 1):
                h = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32", mu=mu))
                x = torch.empty_like(b)
                h.solve(b, x, tol=1e-6, precision="mixed", stream=stream, max_iter=200, raise_on_notconv=False)
                flush.fill_(0.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, st = h.solve(b, x, tol=1e-6, precision="mixed", stream=stream, max_iter=200,
                                raise_on_notconv=False)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                act = (b != 0) | (x != 0)              # inactive cells keep b = x = 0
                rms = lambda e: math.sqrt(float((V[act] * e[act] * e[act]).sum() / V[act].sum()))
                div = (b - h.apply_A(x, stream=stream)) / V
                kh = min(st.iterations, 127)                     # the recorded residual history
                row["mu%d" % mu] = {"iterations": st.iterations, "converged": bool(st.converged),
                                    "rel_res": st.rel_res, "ms": round(ms, 3),
                                    "value": round(g.n_leaves / (ms / 1e3) / 1e6, 3), "unit": UNIT,
                                    "mean_reduction_per_iteration":
                                        round(math.exp(-math.log(st.hist[kh]) / kh), 2),
                                    "fitted_reduction_per_iteration": round(math.exp(-np.polyfit(
                                        np.arange(kh + 1), np.log([st.hist[i] for i in range(kh + 1)]), 1)[0]), 2),
                                    "max_dev_from_y_minus_1": (x - ref)[act].abs().max().item(),
                                    "div_rms_ratio": rms(div) / rms(b / V)}
                del h
            row["solid_cells"] = "inactive (exact fractions)" if inactive else "beta clamped at 1e-3"
            out["%s_%d%s" % (obstacle, n0, "" if inactive else "_clamped")] = row
    return {"cases": out,
            "what": "static tank, mixed solves to 1e-6; with the solid interior at beta 1e-3 the exact "
                    "discrete pressure is y - 1 (the uniform velocity is minus the gradient of a linear "
                    "field); deviations and divergence over the active cells"}


def _accuracy(dev, stream):
    """The paper's accuracy studies (Sec. 4) at root grids 32/64/128: the Laplacian test
    (composite operator in FP64 applied to (x^2+y^2+z^2) exp(-xyz); volume-weighted RMS
    error on the leaves that touch no wall, split into the cells beside a T-junction face
    and the rest) and the sinusoidal Poisson test (FP64 solve to 1e-10 for the solution
    error; mixed solve to 1e-6 for iterations and residual reduction per iteration)."""
    import math
    import numpy as np
    import torch
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S

    def rates(e):
        return [round(math.log2(e[i] / e[i + 1]), 3) for i in range(len(e) - 1)]

    sizes = (32, 64, 128)
    lap = {}
    for kind in ("uniform", "ball", "star"):
        rms, far, tmax = [], [], []
        for n0 in sizes:
            p = P.laplacian_problem(kind, n0)
            g = S.Octree(p.desc)
            f = g.faces()
            h_ = S.Hierarchy(g, P.face_beta(p, f), p.bc, S.mg_params(coef="f64"))
            lv = g.leaves()
            h, x, y, z = P.leaf_centres(n0, lv)
            fv = torch.from_numpy(P.laplacian_test_function(x, y, z)).to(dev)
            e = -h_.apply_A(fv, stream=stream).cpu().numpy() / h ** 3 - P.laplacian_test_exact(x, y, z)
            inner = P.interior_leaves(n0, lv)
            tm = P.t_junction_leaves(g.n_leaves, lv, f)
            rms.append(P.rms_v(h, e, inner))
            far.append(P.rms_v(h, e, inner & ~tm))
            tmax.append(float(np.abs(e[inner & tm]).max()) if np.any(inner & tm) else 0.0)
            del h_
        lap[kind] = {"n0": list(sizes), "rms": rms, "rms_rates": rates(rms), "rms_away_from_t": far,
                     "rates_away_from_t": rates(far), "max_beside_t": tmax}
    sin = {}
    for kind in ("ball", "band", "star"):
        errs, its, red, ms, leaves = [], [], [], [], []
        for n0 in sizes:
            p = P.sinusoidal(kind, n0)
            g = S.Octree(p.desc)
            f = g.faces()
            beta = P.face_beta(p, f)
            lv = g.leaves()
            b = torch.from_numpy(P.rhs(p, lv)).to(dev)
            h64 = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f64"))
            x, st = h64.solve(b, tol=1e-10, precision="fp64", max_iter=60, stream=stream)
            h, xc, yc, zc = P.leaf_centres(n0, lv)
            errs.append(P.rms_v(h, x.cpu().numpy() - P.exact_solution(p, xc, yc, zc)))
            del h64
            h32 = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32"))
            xm = torch.empty_like(b)
            h32.solve(b, xm, tol=1e-6, precision="mixed", stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, sm = h32.solve(b, xm, tol=1e-6, precision="mixed", stream=stream)
            e1.record(stream)
            e1.synchronize()
            its.append(sm.iterations)
            red.append(round(math.exp(-math.log(sm.hist[sm.iterations]) / sm.iterations), 2))
            ms.append(round(e0.elapsed_time(e1), 3))
            leaves.append(g.n_leaves)
            del h32
        sin[kind] = {"n0": list(sizes), "leaves": leaves, "rms_error": errs, "rates": rates(errs),
                     "iterations_1e-6": its, "mean_reduction_per_iteration": red, "ms_mixed_1e-6": ms}
    return {"laplacian": lap, "sinusoidal": sin,
            "grids": "uniform n0^3; ball: refined once within 0.25 of the centre; band: refined twice "
                     "within 0.05 of the sphere r = 0.25; star: refined twice where cells meet the star "
                     "surface r = 0.237 + 0.079 cos(6 theta) cos(6 phi)"}


def _large(dev, stream, flush, args, peak):
    """The sine-band workload at full size: mixed solve to 1e-6 (timed), the red-black sweep
    on its finest level (per-launch events inside an unrolled graph of the same solve),
    and the adjoint (transpose solve + face gradient)."""
    import numpy as np
    import torch
    from paper_2604_18886_b300 import _lib as L
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S
    t0 = time.perf_counter()
    p = P.sine_band(args.large_n0, 3)
    g = S.Octree(p.desc)
    t_build = time.perf_counter() - t0
    beta, bh = P.large_inputs(p, g.n_leaves, g.n_faces, g.faces_range, dev)
    b = torch.from_numpy(bh).to(dev)
    del bh
    t1 = time.perf_counter()
    h = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32", sweep=args.sweep))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t1
    x = torch.empty_like(b)
    for _ in range(args.warmup):
        h.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
    steps = max(1 if args.only_large else 3, min(args.steps, 10))
    t, its = [], set()
    for s_ in range(steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if args.nvtx:
            torch.cuda.nvtx.range_push("timed")
        _, st = h.solve(b, x, tol=1e-6, precision="mixed", stream=stream, eager=args.eager)
        if args.nvtx:
            torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        t.append(e0.elapsed_time(e1))
        its.add(st.iterations)
        assert st.converged
    ms = statistics.mean(t)
    tun = h.tuning()
    forms = {str(m): {"form": S.SWEEP_FORM_NAMES.get(v[0], "shared-memory tail"), "us_octet": round(v[1], 2),
                      "us_cell": round(v[2], 2), "us_quad": round(v[3], 2), "us_tile": round(v[4], 2)}
             for m, v in tun.items() if m >= 0}
    if args.only_large:
        out = {"workload": LARGE_WORKLOAD, "n0": args.large_n0, "leaves": g.n_leaves,
               "value": round(g.n_leaves / (ms / 1e3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms, 3),
               "steps": steps, "iterations": sorted(its), "sweep_forms": forms,
               "note": "--only-large (profiling aid)"}
        if args.adjoint:
            # one transpose solve (tables built and graph captured by an untimed first call),
            # then one more inside the NVTX range 'adjoint' (kernel by kernel with --eager)
            gp = x - torch.from_numpy(np.random.default_rng(8).standard_normal(g.n_leaves)).to(dev)
            h.solve(gp, tol=1e-6, precision="mixed", stream=stream, transpose=True, max_iter=200)
            torch.cuda.synchronize()
            if args.nvtx:
                torch.cuda.nvtx.range_push("adjoint")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, sa = h.solve(gp, tol=1e-6, precision="mixed", stream=stream, transpose=True, max_iter=200,
                            eager=args.eager)
            e1.record(stream)
            e1.synchronize()
            if args.nvtx:
                torch.cuda.nvtx.range_pop()
            out["adjoint"] = {"ms": round(e0.elapsed_time(e1), 3), "iterations": sa.iterations}
        return out
    # plain FP32 beside it (FP32 Krylov vectors, FP64 dot products)
    t32 = []
    for s_ in range(steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st32 = h.solve(b, x, tol=1e-6, precision="fp32", stream=stream)
        e1.record(stream)
        e1.synchronize()
        t32.append(e0.elapsed_time(e1))
    ms32 = statistics.mean(t32)
    wc = _w_cycle(g, beta, p, b, dev, stream, flush, steps)
    wh = _w_cycle(g, beta, p, b, dev, stream, flush, steps, mu_min_cells=HYBRID_MIN_CELLS)
    # finest-level sweep inside an unrolled graph of the same solve
    D = g.D
    L.check(L.lib().ocg_probe_set(h.handle, L.OCG_PROBE_SWEEP, D))
    h.solve(b, x, tol=1e-6, precision="mixed", stream=stream, max_iter=st.iterations, unrolled=True,
            raise_on_notconv=False)
    nl, tot, ce = C.c_int64(), C.c_double(), C.c_int64()
    L.check(L.lib().ocg_probe_read(h.handle, C.c_void_p(stream.cuda_stream), C.byref(nl), C.byref(tot),
                                   C.byref(ce)))
    L.check(L.lib().ocg_probe_set(h.handle, L.OCG_PROBE_OFF, 0))
    sweep_us = tot.value * 1e3 / max(nl.value, 1)
    achieved = SWEEP_BYTES_PER_CELL * ce.value / (sweep_us / 1e6) / 1e9
    form = S.SWEEP_FORM_NAMES.get(tun[D][0], "?")
    # adjoint: transpose solve of dL/dp = p - p_t and the face gradient
    ptgt = torch.from_numpy(np.random.default_rng(8).standard_normal(g.n_leaves)).to(dev)
    gp = x - ptgt
    del ptgt
    def adjoint(hier, method="pcg"):
        # the first call builds the adjoint tables and captures the graph: untimed
        res = []
        for r in range(2):
            flush.fill_(float(r))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lam, sa = hier.solve(gp, tol=1e-6, precision="mixed", stream=stream, transpose=True, max_iter=200,
                                 raise_on_notconv=False, method=method)
            hier.face_grad(x, lam, stream=stream)
            e1.record(stream)
            e1.synchronize()
            res.append((e0.elapsed_time(e1), sa))
        return res[-1]

    ms_a, sa = adjoint(h)
    adj = {"ms": round(ms_a, 3), "iterations": sa.iterations, "converged": bool(sa.converged),
           "rel_res": sa.rel_res,
           "what": "A^T lambda = p - p_t by Alg. 1 on A^T preconditioned by M^T (mixed, tol 1e-6) + face "
                   "gradient; second call (the first builds the adjoint tables and the graph)"}
    ms_b, sb = adjoint(h, "bicgstab")
    adj["bicgstab"] = {"ms": round(ms_b, 3), "iterations": sb.iterations, "converged": bool(sb.converged)}
    # the same adjoint preconditioned by the hybrid cycle
    hh = S.Hierarchy(g, beta, p.bc, S.mg_params(mu=2, coef="f32", mu_min_cells=HYBRID_MIN_CELLS))
    ms_h, sh_ = adjoint(hh)
    adj["hybrid_cycle"] = {"ms": round(ms_h, 3), "iterations": sh_.iterations, "converged": bool(sh_.converged)}
    del hh
    return {"workload": LARGE_WORKLOAD, "leaves": g.n_leaves, "faces": g.n_faces, "cells_all_levels": g.n_cells,
            "precision": "mixed (FP32 V-cycle, FP64 PCG)", "value": round(g.n_leaves / (ms / 1e3) / 1e6, 3),
            "unit": UNIT, "ms_per_step": round(ms, 3), "steps": steps, "iterations": sorted(its),
            "true_rel_res": st.true_rel_res, "build_s": round(t_build, 2), "setup_s": round(t_setup, 2),
            "w_cycle": wc, "w_v_hybrid": wh,
            "plain_fp32": {"value": round(g.n_leaves / (ms32 / 1e3) / 1e6, 3), "unit": UNIT,
                           "ms_per_step": round(ms32, 3), "iterations": st32.iterations,
                           "true_rel_res": st32.true_rel_res},
            "sweep_forms": forms,
            "roofline": {"bound": "hbm", "kernel": "red-black colour sweep (%s form) on level %d" % (form, D),
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                         "bytes_per_cell": SWEEP_BYTES_PER_CELL,
                         "cells_per_launch": ce.value, "launches": nl.value, "avg_launch_us": round(sweep_us, 2),
                         "traffic": _profiled_traffic("sweep_sineband_level%d_%s" % (D, form), ce.value),
                         "traffic_note": "dram bytes per cell of an ncu capture at 64^3 root (same field, "
                                         "effective 512^3) times the cells of one launch"},
            "adjoint": adj}


BATCH_WORKLOAD = ("64 independent octrees, effective 64/96/128 with 2-3 levels refined within 0.05 of a "
                  "seeded random sphere; even trees beta=1 Dirichlet, odd trees cut-cell beta Neumann; "
                  "rhs N(0,1)")


def _batched(dev, stream, flush, args):
    """The batched workload solved by ocg_pcg_solve_batched, and the same 64 problems
    solved one after another by single graph solves, both mixed precision to 1e-6."""
    import torch
    from paper_2604_18886_b300 import problems as P
    from paper_2604_18886_b300 import solver as S
    hs, bs, leaves = [], [], 0
    for k in range(64):
        p = P.batch_tree(k)
        g = S.Octree(p.desc)
        f = g.faces()
        beta = P.face_beta(p, f)
        hs.append(S.Hierarchy(g, torch.from_numpy(beta).to(dev), p.bc, S.mg_params(coef="f32")))
        bs.append(torch.from_numpy(P.rhs(p, g.leaves(), f, beta)).to(dev))
        leaves += g.n_leaves
    t0 = time.perf_counter()
    bt = S.Batch(hs, stream=stream)
    t_create = time.perf_counter() - t0
    xs = [torch.empty_like(b) for b in bs]
    for _ in range(args.warmup):
        bt.solve(bs, xs, tol=1e-6, stream=stream)
    steps = max(3, min(args.steps, 20))
    tb, its, kern = [], set(), 0
    for s_ in range(steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = bt.solve(bs, xs, tol=1e-6, stream=stream)
        e1.record(stream)
        e1.synchronize()
        tb.append(e0.elapsed_time(e1))
        its.update(x.iterations for x in st)
        kern += st[0].kernels
        assert all(x.converged for x in st)
    # the same problems one after another (single graph solves)
    for h, b, x in zip(hs, bs, xs):
        h.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
    ts = []
    for s_ in range(3):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h, b, x in zip(hs, bs, xs):
            h.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms_b = statistics.mean(tb)
    ms_s = statistics.mean(ts)
    forms = {str(h): ["octet", "cell"][f] for h, (f, a, b) in bt.info().items()}
    del bt
    return {"workload": BATCH_WORKLOAD, "problems": 64, "leaves": leaves,
            "value": round(leaves / (ms_b / 1e3) / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms_b, 4),
            "steps": steps, "iterations": sorted(its), "gpu_launches_per_step": kern // steps,
            "sweep_forms_by_height": forms, "create_s": round(t_create, 3),
            "sequential_single_solves": {"value": round(leaves / (ms_s / 1e3) / 1e6, 3), "unit": UNIT,
                                         "ms_per_step": round(ms_s, 4)}}


def _time_solves(hier, b, x, steps, precision, flush, stream, nvtx=False, eager=False):
    import torch
    times, iters, kernels = [], [], 0
    for s in range(steps):
        flush.fill_(float(s))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if nvtx:
            torch.cuda.nvtx.range_push("timed")
        _, st = hier.solve(b, x, tol=1e-6, precision=precision, stream=stream, eager=eager)
        if nvtx:
            torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        iters.append(st.iterations)
        kernels += st.kernels
        assert st.converged
    return times, iters, kernels


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2604_18886_b300 import _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.only_large:
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        out = _large(dev, stream, flush, args, _peaks()[0])
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    p, tree, hier, b, np = _setup(dev, args.headline_sweep)
    x = torch.empty_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(args.warmup):
        hier.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
        hier.solve(b, x, tol=1e-6, precision="fp32", stream=stream)
    # ---- timed region: mixed solve (graph path, one host synchronisation per solve)
    levels = [tree.level(m)[0].shape[0] for m in range(0, tree.D + 1)]
    big = int(max(range(len(levels)), key=lambda q: levels[q]))
    clocks = Clocks(local)
    clocks.wait_first()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    mark0 = clocks.mark()
    t0 = time.perf_counter()
    times, iters, kernels = _time_solves(hier, b, x, args.steps, "mixed", flush, stream, nvtx=args.nvtx,
                                         eager=args.eager)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    mark1 = clocks.mark()
    if world > 1:
        dist.barrier()
    ck = clocks.stop(mark0, mark1)
    ms = statistics.mean(times)
    total_ms = sum(times)
    from paper_2604_18886_b300 import solver as S
    tuning = {str(m): {"form": S.SWEEP_FORM_NAMES[f] if f >= 0 else "shared-memory tail",
                       "us_octet": round(a, 2), "us_cell": round(bq, 2), "us_quad": round(qq, 2),
                       "us_tile": round(tt, 2)}
              for m, (f, a, bq, qq, tt) in hier.tuning().items()}
    total_ms = max_over_ranks(total_ms, dev)
    value = replica_throughput(tree.n_leaves, args.steps, world, total_ms)
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 3), "unit": UNIT, "steps": args.steps,
                              "ms_per_step": round(ms, 4), "note": "--only-timed (profiling aid)"}), flush=True)
        return
    # ---- per-kernel durations inside a graph: the same solve (same iteration count) as
    # one flat graph whose probe events are event-record nodes around the probed launches
    def probe(kind, level, reps=5):
        L.check(L.lib().ocg_probe_set(hier.handle, kind, level))
        nl_t, ms_t, cells = 0, 0.0, 0
        for r in range(reps):
            flush.fill_(float(r))
            hier.solve(b, x, tol=1e-6, precision="mixed", stream=stream, max_iter=iters[0], unrolled=True,
                       raise_on_notconv=False)
            nl, tot, ce = C.c_int64(), C.c_double(), C.c_int64()
            L.check(L.lib().ocg_probe_read(hier.handle, C.c_void_p(stream.cuda_stream), C.byref(nl),
                                           C.byref(tot), C.byref(ce)))
            nl_t += nl.value
            ms_t += tot.value
            cells = ce.value
        L.check(L.lib().ocg_probe_set(hier.handle, L.OCG_PROBE_OFF, 0))
        return nl_t, ms_t, cells
    sw_n, sw_ms, sw_cells = probe(L.OCG_PROBE_SWEEP, big)
    tail_top = max([m for m, v in hier.tuning().items() if v[0] < 0 and m < 0] or [tree.mc])
    tl_n, tl_ms, tl_cells = probe(L.OCG_PROBE_TAIL, tail_top)
    ap_n, ap_ms, ap_cells = probe(L.OCG_PROBE_APPLY, 0)
    # ---- plain FP32 beside it
    times32, iters32, _ = _time_solves(hier, b, x, args.steps, "fp32", flush, stream)
    v32 = tree.n_leaves / (statistics.mean(times32) / 1e3) / 1e6
    # ---- mixed with BF16 coarse-level coefficients
    hb = _hier_bf16(p, tree, dev)
    for _ in range(args.warmup):
        hb.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
    times_b, iters_b, _ = _time_solves(hb, b, x, args.steps, "mixed", flush, stream)
    vb16 = tree.n_leaves / (statistics.mean(times_b) / 1e3) / 1e6
    del hb
    # ---- adjoint: transpose solve (Alg. 1 on A^T, transposed cycle M^T) + face gradient
    ptgt = torch.from_numpy(np.random.default_rng(2).standard_normal(tree.n_leaves)).to(dev)
    xs, _ = hier.solve(b, tol=1e-6, precision="mixed", stream=stream)
    gp = xs - ptgt
    adj_t, adj_it = [], []
    for r in range(max(3, min(args.steps, 20))):
        flush.fill_(float(r))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam, sa = hier.solve(gp, tol=1e-6, precision="mixed", stream=stream, transpose=True)
        hier.face_grad(xs, lam, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if r > 0:
            adj_t.append(e0.elapsed_time(e1))
            adj_it.append(sa.iterations)
    # ---- cut-cell workload (mixed, BF16 coarse coefficients)
    cut = None if args.no_batch else _cut_cell(dev, stream, flush, args)
    # ---- batched form: 64 independent trees, one graph, one launch per phase
    batched = None if args.no_batch else _batched(dev, stream, flush, args)
    # ---- the large sine-band workload (effective 1024^3)
    large = None if args.no_large else _large(dev, stream, flush, args, _peaks()[0])
    accuracy = None if args.no_accuracy else _accuracy(dev, stream)
    tank = None if args.no_accuracy else _tank(dev, stream, flush, args)
    # ---- end to end through the C ABI with host buffers
    bh = b.cpu().pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    e2e_t = []
    for s_ in range(args.steps):
        flush.fill_(float(s_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.copy_(bh, non_blocking=True)
        hier.solve(b, x, tol=1e-6, precision="mixed", stream=stream)
        xh.copy_(x, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_t.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_t), dev)
    e2e = replica_throughput(tree.n_leaves, args.steps, world, e2e_total)
    # ---- roofline of the dominant kernel family: the red-black sweep on the largest level
    peak, peak_kind = _peaks()
    sweep_us = sw_ms * 1e3 / max(sw_n, 1)
    achieved = SWEEP_BYTES_PER_CELL * sw_cells / (sweep_us / 1e6) / 1e9
    fwd = tuning.get(str(big), {}).get("form", "octet")
    traffic = _profiled_traffic("sweep_ball64_level%d_%s" % (big, fwd), sw_cells)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 cycle + f64 pcg", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "mixed (FP32 V-cycle, FP64 PCG)", "tol": 1e-6,
                   "leaves": tree.n_leaves, "iterations": sorted(set(iters)),
                   "cycle": "V (mu=1), nu=2/2, coarsest 10",
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "sweep_forms": tuning,
                   "wall_s_timed": round(wall, 3)},
        "plain_fp32": {"value": round(v32, 3), "unit": UNIT, "ms_per_step": round(statistics.mean(times32), 4),
                       "iterations": sorted(set(iters32))},
        "mixed_bf16_coarse": {"value": round(vb16, 3), "unit": UNIT,
                              "ms_per_step": round(statistics.mean(times_b), 4),
                              "iterations": sorted(set(iters_b))},
        "adjoint": {"ms": round(statistics.mean(adj_t), 4), "iterations": sorted(set(adj_it)),
                    "what": "A^T lambda = p - p_t by Alg. 1 on A^T preconditioned by M^T (mixed, tol 1e-6) "
                            "+ face gradient"},
        "value_mi_cells": round(value / 1.048576, 3),
        "roofline": {"bound": "hbm", "kernel": "red-black colour sweep (%s form) on level %d" % (fwd, big),
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                     "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "bytes_per_cell": SWEEP_BYTES_PER_CELL, "cells_per_launch": sw_cells,
                     "launches": sw_n, "avg_launch_us": round(sweep_us, 3),
                     "timing": "CUDA event-record nodes around each launch inside one graph of the solve",
                     "traffic": traffic},
        "kernels_us": {"coarse_tail": round(tl_ms * 1e3 / max(tl_n, 1), 3), "coarse_tail_launches": tl_n,
                       "operator_apply": round(ap_ms * 1e3 / max(ap_n, 1), 3), "operator_launches": ap_n},
        "cut_cell": cut,
        "batched": batched,
        "large": large,
        "accuracy": accuracy,
        "tank": tank,
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": tree.n_leaves * 8,
                "d2h_bytes_per_step": tree.n_leaves * 8},
        "clocks": ck,
        "gpu_launches": int(kernels),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _oracle_problem():
    from oracle import octree as O
    from oracle import operator as OP
    from paper_2604_18886_b300 import problems as P
    p = P.two_level_ball(64)
    t = O.Octree(p.desc)
    f = t.faces()
    beta = P.face_beta(p, f)
    H = OP.Hierarchy(t, beta, p.bc)
    b = P.rhs(p, t.leaves, f, beta)
    return t, H, b


def cpu_baseline(budget_s=15.0):
    """The FP64 oracle (explicit CSR, scipy) timed on the host on the same workload."""
    from oracle import pcg
    t, H, b = _oracle_problem()
    times = []
    t_end = time.perf_counter() + budget_s
    while not times or (time.perf_counter() < t_end and len(times) < 20):
        t0 = time.perf_counter()
        pcg.pcg(H, b, tol=1e-6)
        times.append(time.perf_counter() - t0)
    v = t.n_leaves / statistics.mean(times) / 1e6
    return {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full solves of the same workload (oracle set-up excluded), %.1f s" %
                      (len(times), sum(times))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import pcg
    t, H, b = _oracle_problem()
    for _ in range(args.warmup):
        pcg.pcg(H, b, tol=1e-6)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, k, _ = pcg.pcg(H, b, tol=1e-6)
        times.append(time.perf_counter() - t0)
    ms = statistics.mean(times) * 1e3
    v = t.n_leaves / (ms / 1e3) / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "FP64 oracle (scipy CSR, Alg. 4 cycle, Alg. 1)",
                      "tol": 1e-6, "leaves": t.n_leaves, "iterations": k},
           "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "one full solve per step (set-up excluded)"},
           "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--nvtx", action="store_true", help="NVTX range 'timed' around the timed mixed solves")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-tree form")
    ap.add_argument("--no-large", action="store_true", help="skip the large sine-band workload")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy studies and the static tank")
    ap.add_argument("--only-large", action="store_true",
                    help="run only the timed solves of the large sine-band workload (profiling aid)")
    ap.add_argument("--sweep", default="auto", choices=["auto", "octet", "cell", "quad", "tile"],
                    help="sweep form of the large workload's hierarchy (auto: timed at set-up; profiling aid)")
    ap.add_argument("--large-n0", type=int, default=128,
                    help="root grid of the sine-band workload (128: effective 1024^3; smaller for profiling)")
    ap.add_argument("--only-timed", action="store_true",
                    help="run the warm-up and the timed mixed solves only (profiling aid)")
    ap.add_argument("--eager", action="store_true",
                    help="launch the timed solves kernel by kernel (profiling aid; not the benchmark path)")
    ap.add_argument("--headline-sweep", default="auto", choices=["auto", "octet", "cell", "quad", "tile"],
                    help="sweep form of the headline hierarchy (auto: timed at set-up; profiling aid)")
    ap.add_argument("--adjoint", action="store_true",
                    help="with --only-large: also one transpose solve, in the NVTX range 'adjoint' (profiling aid)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
