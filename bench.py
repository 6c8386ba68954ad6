#!/usr/bin/env python
"""Benchmark: G-column solves/s of the real-space NEGF transmission path.

Workload (one "step"): the 24x24x120 synthetic molecular junction (69,120
points, h = 0.35 bohr, 8th-order FD, soft-square leads, 20 Gaussian wells, 20
atoms x 4 s/p KB projectors, 8-plane quadratic CAP, seed 1) at one energy from
128 in [0.16, 0.24] Ha: the partial T(E) and dT(E)/dV_loc over a batch of 288
right-CAP columns (every 16th of the 4,608).  Each column is one unit of the
metric and costs two solves: its forward COCG solve x_j = G e_j and its
adjoint solve lambda_j = G (Gamma_L o conj x_j).  FP32 Krylov recurrence with
FP64 reliable updates to a true relative residual of 1e-10, FP64 T and
gradient sums.

Beside the timed steps the JSON line carries
  * ``roofline``: the COCG operator kernel timed with CUDA events in a separate
    pass over the same energies (no events inside the timed region);
  * ``forward_T``: T(E) alone over 1,152 right-CAP columns (every 4th) at six
    seeded energies of the window, mixed precision and FP64 on the same columns,
    with |dT| and relative dT per energy and the window-averaged speed ratio;
  * ``parity``: T and per-column contributions of 16 golden columns at three
    energies against the oracle's sparse-LU values (tests/golden);
  * ``e2e``: the step through the public API from host buffers (potential in,
    T and dV out) over the timed steps' energies;
  * ``cpu_baseline``: the oracle on columns and energies of the timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank solves its own energies (weak scaling, no
data-path collective); the timed region is bracketed by a barrier and
synchronisation, and rank 0 prints one JSON line with the max over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G-column solves/s, FP32+refine vs FP64 at |ΔT|≤1e-6; matvec HBM GB/s vs peak"
UNIT = "solves/s"
N_ENERGIES = 128
E_LO, E_HI = 0.16, 0.24
WORKLOAD = ("junction 24x24x120 (N=69,120), h=0.35, 8th-order FD, 20 atoms x 4 KB projectors, "
            "8-plane quadratic CAP, seed 1; mixed precision (complex FP32 COCG + FP64 refinement to 1e-10); "
            "one unit = one right-CAP column with its forward and adjoint solve")
CPU_SAMPLE_RTOL = 1e-10
GOLDEN = os.path.join(ROOT, "tests", "golden", "junction_24x24x120_tc.txt")

# DRAM bytes per algorithmic byte of the COCG operator kernel, from one ncu
# capture of the kernel micro-benchmark (python -m paper_1401_0782_gb300.kernel_bench
# --kind op --slots 256 --reps 3): dram__bytes_read.sum + dram__bytes_write.sum
# = 593.3 MB over 32 B x 69,120 points x 256 systems = 566.2 MB.  Retaken
# whenever that kernel changes.
OP_DRAM_PER_ALG_BYTE = 593.25952 / 566.23104


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [num(r[3]) for r in self.rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def dist_init():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist, rank, local, world
    return None, rank, local, world


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def energy_index(rank: int, world: int, k: int) -> int:
    """Grid index of the energy of step k on `rank`: ranks take disjoint
    energies, and consecutive steps stride across the whole window (37 is
    coprime to 128, so the first 128 steps of all ranks never repeat one)."""
    return ((rank + k * world) * 37) % N_ENERGIES


def energy_for(rank: int, world: int, k: int) -> float:
    import numpy as np
    E = np.linspace(E_LO, E_HI, N_ENERGIES)
    return float(E[energy_index(rank, world, k)])


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample; spawn pool, never forked after CUDA init)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    """Forward + adjoint solve of one column by the oracle's Krylov route."""
    col, E, rtol = args
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1401_0782_gb300 import problems as P
    import numpy as np
    j = P.molecular_junction(seed=1)
    t0 = time.perf_counter()
    # the steps of the oracle's transmission_grad at the bench tolerance:
    # forward column, then the adjoint with the same operator
    X, solver = O.solve_columns(j, E, [col], return_lu=True, method="krylov", rtol=rtol)
    solver.solve(j.gamma_l[:, None] * np.conj(X))
    return time.perf_counter() - t0


def oracle_sample(pairs, cores: int):
    """Forward + adjoint oracle solves of the (column, energy) pairs over `cores`
    spawn processes; returns (columns/s, wall seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    # one thread per worker process: the pool, not BLAS, uses the cores
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(pairs[0][0], pairs[0][1], 1e-2)] * cores)  # import + setup warm-up, not timed
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [(c, E, CPU_SAMPLE_RTOL) for c, E in pairs])
        wall = time.perf_counter() - t0
    return len(pairs) / wall, wall


def sample_pairs(cols, energies, n):
    """n (column, energy) pairs: columns of the step's set, cycling over the energies."""
    import numpy as np
    rng = np.random.default_rng(8)
    pick = rng.choice(cols, n, replace=False)
    return [(int(c), float(energies[i % len(energies)])) for i, c in enumerate(pick)]


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def load_golden():
    """{energy index: (E, cols, t_c)} from the oracle-written golden file, or None."""
    import numpy as np
    if not os.path.exists(GOLDEN):
        return None
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    out = {}
    for k, E, c, t, _ in rows:
        out.setdefault(int(k), (float(E), [], []))
        out[int(k)][1].append(int(c))
        out[int(k)][2].append(float(t))
    return {k: (E, np.array(c, np.int32), np.array(t)) for k, (E, c, t) in out.items()}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def passes_per_iteration(j):
    """Algorithmic vector passes (one complex vector of N points read or written
    once) per COCG iteration of one system, by kernel."""
    import numpy as np
    cnt = np.zeros(j.N, np.int64)
    atoms = {}
    for p in range(j.n_proj):
        idx = j.proj_idx[j.proj_offsets[p]:j.proj_offsets[p + 1]]
        atoms.setdefault(idx.tobytes(), idx)
    for idx in atoms.values():
        cnt[idx] += 1
    gath = float(cnt.sum()) / j.N
    # the projector term of q is added inside the update kernel (q is read once
    # there anyway and never written back), so it costs no vector pass
    d = {"operator": 4.0, "update": 6.0, "r_projection": gath}
    d["total"] = sum(d.values())
    d["floor"] = 6.0
    d["launches_per_iteration"] = 11
    return d


def run_ours(args):
    import numpy as np
    import torch

    from paper_1401_0782_gb300 import binding as B
    from paper_1401_0782_gb300 import problems as P

    dist, rank, local, world = dist_init()
    torch.cuda.set_device(local)
    j = P.molecular_junction(seed=1)
    all_cols = j.right_columns()
    cols = all_cols
    if args.cols_per_step and args.cols_per_step < cols.size:
        cols = cols[:: int(np.ceil(cols.size / args.cols_per_step))]
    n_cols = int(cols.size)
    ctx = B.Context(local).set_junction(j)
    opts = B.default_opts(B.RSN_MIXED, deadline_ms=args.deadline * 1e3)
    # operator-kernel tile for this grid and slot count (untimed set-up)
    tuned = ctx.autotune(B.RSN_MIXED, min(2048, max(256, 2 * n_cols // 4)))
    print(f"[bench] autotuned tile {tuned}", file=sys.stderr, flush=True)
    dV = torch.empty(j.N, dtype=torch.float64, device=f"cuda:{local}")

    def step(k, o):
        E = energy_for(rank, world, k)
        T, _ = ctx.transmission_vjp([E], [1.0], cols, o, dV_out=dV)
        return T

    t_w = time.perf_counter()
    for k in range(args.warmup):
        step(k, opts)
        print(f"[bench] warm-up step {k}: {time.perf_counter() - t_w:.1f} s {ctx.last_stats()}", file=sys.stderr,
              flush=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    t_wall = time.perf_counter()
    launches = iters = fallbacks = 0
    step_stats = []
    timed = list(range(args.warmup, args.warmup + args.steps))
    for k in timed:
        step(k, opts)
        st = ctx.last_stats()
        launches += st["launches"]
        iters += st["krylov_iters"]
        fallbacks += st["fp64_fallbacks"]
        step_stats.append((k, st))
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks.stop()
    for k, st in step_stats:
        print(f"[bench] step {k} E={energy_for(rank, world, k):.5f}: {st}", file=sys.stderr, flush=True)
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(dist, ms)
    total_units = sum_over_ranks(dist, float(args.steps * n_cols))
    value = total_units / (ms_max / 1e3)

    # ---- roofline: the operator kernel timed with events in its own pass -----
    ot = B.default_opts(B.RSN_MIXED, deadline_ms=args.deadline * 1e3, timing=1)
    kb = kms = 0.0
    klaunch = 0
    ub = ums = 0.0
    for k in timed[: max(1, min(len(timed), args.roofline_steps))]:
        step(k, ot)
        s0, s1 = ctx.kernel_stats(0), ctx.kernel_stats(1)
        kb += s0["bytes"]
        kms += s0["ms"]
        klaunch += s0["launches"]
        ub += s1["bytes"]
        ums += s1["ms"]

    # ---- end to end through the public API with host buffers -------------
    # every step uploads its potential (host -> device, the input of T and
    # dT/dV_loc) and reads T and dV back; energies of the timed steps
    e2e_ks = [timed[i % len(timed)] for i in range(max(5, len(timed)))]
    v_host = np.ascontiguousarray(j.v_loc, dtype=np.float64)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    te = time.perf_counter()
    for k in e2e_ks:
        ctx.set_potential(v_host)
        T_h, dV_h = ctx.transmission_vjp([energy_for(rank, world, k)], [1.0], cols, opts)
    e2e_s = max_over_ranks(dist, time.perf_counter() - te)
    e2e_value = sum_over_ranks(dist, float(len(e2e_ks) * n_cols)) / e2e_s
    h2d = v_host.nbytes + 8 + 8 + cols.nbytes
    d2h = dV_h.nbytes + T_h.nbytes

    result = None
    if rank == 0:
        peak, peak_kind = measured_peaks()
        achieved = kb / (kms / 1e3) / 1e9 if kms > 0 else None
        upd = ub / (ums / 1e3) / 1e9 if ums > 0 else None
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": {
                "workload": WORKLOAD, "grid": [j.nx, j.ny, j.nz], "N": j.N, "fd_order": 2 * j.fd_half_order,
                "n_proj": j.n_proj, "columns_per_step": n_cols, "solves_per_step": 2 * n_cols,
                "unit_definition": "one right-CAP column j: forward solve x_j = G e_j and adjoint solve "
                                   "lambda_j = G (Gamma_L o conj x_j), both to true relative residual 1e-10",
                "step": "partial T(E) + dT/dV_loc at one energy over every 16th right-CAP column",
                "energies": f"step k on rank r: E[37 (r + k*world) mod {N_ENERGIES}] of linspace({E_LO},{E_HI},{N_ENERGIES})",
                "tol": opts.tol, "tol_inner": opts.tol_inner,
                "l2": "inputs larger than L2: per-step working set "
                      f"{(j.N * 2 * n_cols * (16 + 16 + 5 * 8)) / 1e9:.1f} GB",
                "parallelism": f"replicas x{world}: energies sharded over ranks, no collective in the data path",
                "tile": tuned,
            },
            "roofline": {
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": (OP_DRAM_PER_ALG_BYTE * kb / klaunch) if (klaunch and OP_DRAM_PER_ALG_BYTE) else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per algorithmic byte of one "
                                  "kernel_bench launch (256 slots), scaled to this run's mean launch",
                "kernel": "op_pair_kernel<4,OP_COCG> (p = r + beta p_old, 25-point stencil + V/CAP on point "
                          "pairs with bulk-copied planes, p^T A p); the projector term of A p is added on the "
                          "support points inside the update kernel",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                               "fallback 6.8 TB/s",
                "algorithmic_bytes": "32 B per active system per grid point (read r, p_old; write p_new, q)",
                "timing": f"CUDA events around every operator launch on the library stream, in a separate pass "
                          f"over the first {max(1, min(len(timed), args.roofline_steps))} timed steps' energies",
                "launches_timed": klaunch, "kernel_ms": kms, "mean_launch_bytes": kb / klaunch if klaunch else None,
                "update_kernel_gbs": upd,
                "update_kernel_note": "COCG update with the support-point projector term, 6 vectors x 8 B per point "
                                      "algorithmic",
            },
            "passes_per_iteration": passes_per_iteration(j),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "steps": len(e2e_ks), "energies": "those of the timed steps (cycled to at least five)",
                    "per_step": "set_potential (host V_loc) + transmission_vjp with host T and dV"},
            "gpu_launches": int(launches),
            "krylov_iters_per_solve": iters / float(args.steps * 2 * n_cols),
            "fp64_fallback_solves": int(fallbacks),
            "clocks": clocks.summary(),
            "wall_s": wall,
        }

    # ---- forward T over every right-CAP column: mixed against FP64 ----------
    if rank == 0 and not args.no_fp64:
        rng = np.random.default_rng(17)
        E_grid = np.linspace(E_LO, E_HI, N_ENERGIES)
        eidx = sorted(rng.choice(N_ENERGIES, args.fwd_energies, replace=False).tolist())
        fcols = all_cols[:: max(1, all_cols.size // args.fwd_cols)] if args.fwd_cols else all_cols
        per_e = []
        tm_tot = t64_tot = 0.0
        for i in eidx:
            E = float(E_grid[i])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Tm = ctx.transmission([E], fcols, B.default_opts(B.RSN_MIXED))[0]
            tm = time.perf_counter() - t0
            sm = ctx.last_stats()
            t0 = time.perf_counter()
            T64 = ctx.transmission([E], fcols, B.default_opts(B.RSN_FP64))[0]
            t64 = time.perf_counter() - t0
            s64 = ctx.last_stats()
            tm_tot += tm
            t64_tot += t64
            per_e.append({"E": E, "T_mixed": float(Tm), "T_fp64": float(T64), "abs_dT": float(abs(Tm - T64)),
                          "rel_dT": float(abs(Tm - T64) / abs(T64)) if T64 else None,
                          "mixed_s": tm, "fp64_s": t64,
                          "iters_per_solve_mixed": sm["krylov_iters"] / fcols.size,
                          "iters_per_solve_fp64": s64["krylov_iters"] / fcols.size,
                          "fp64_fallbacks": sm["fp64_fallbacks"]})
        n = fcols.size * len(eidx)
        result["forward_T"] = {
            "sample": f"{fcols.size} right-CAP columns x energies {eidx} of linspace({E_LO},{E_HI},{N_ENERGIES}); "
                      "forward solves only, host-timed library calls",
            "mixed_solves_per_s": n / tm_tot, "fp64_solves_per_s": n / t64_tot,
            "mixed_over_fp64": t64_tot / tm_tot, "per_energy": per_e,
            "note": "T ~ 1e-19..1e-13 in this window (every lead channel is closed), so |dT| <= 1e-6 is met by "
                    "construction; rel_dT is the meaningful figure",
        }

    # ---- an energy window by shifted COCG against one solve per energy ----
    if rank == 0 and not args.no_fp64 and args.window_energies > 0:
        E_win = np.linspace(E_LO, E_HI, args.window_energies)
        wcols = all_cols[:: max(1, all_cols.size // args.window_cols)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ts, its = ctx.transmission_shifted(E_win, wcols, B.default_opts(B.RSN_FP64), return_iters=True)
        ts = time.perf_counter() - t0
        ss = ctx.last_stats()
        t0 = time.perf_counter()
        Tm = ctx.transmission(E_win, wcols, B.default_opts(B.RSN_MIXED))
        tm = time.perf_counter() - t0
        sm = ctx.last_stats()
        n = E_win.size * wcols.size
        result["window_T"] = {
            "sample": f"{wcols.size} right-CAP columns x {E_win.size} energies linspace({E_LO},{E_HI}); host-timed",
            "shifted_fp64_solves_per_s": n / ts, "per_energy_mixed_solves_per_s": n / tm,
            "shifted_over_mixed": tm / ts,
            "seed_iterations_max": int(its.max()), "operator_applications_shifted": ss["krylov_iters"],
            "operator_applications_per_energy_mixed": sm["krylov_iters"],
            "max_rel_dT_shifted_vs_mixed": float(np.max(np.abs(Ts - Tm) / np.abs(Ts))),
            "plain_fp64_fallbacks": ss["fp64_fallbacks"],
        }

    # ---- block COCG: the columns of one energy share one Krylov space ------
    if rank == 0 and not args.no_fp64 and args.block_cols > 0:
        E_blk = np.linspace(E_LO, E_HI, N_ENERGIES)[[37, 101]]
        kcols = all_cols[:: max(1, all_cols.size // args.block_cols)]
        om = B.default_opts(B.RSN_MIXED, deadline_ms=args.deadline * 1e3)
        leg = {"sample": f"{kcols.size} right-CAP columns x energies {E_blk.round(5).tolist()}; forward T, host-timed "
                         "library calls, both paths on the same systems"}
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Tm = ctx.transmission(E_blk, kcols, om)
            tm = time.perf_counter() - t0
            sm = ctx.last_stats()
            n = E_blk.size * kcols.size
            leg["plain_mixed_solves_per_s"] = n / tm
            leg["plain_mixed_iters_per_solve"] = sm["krylov_iters"] / n
            for blk in (16, 8):
                t0 = time.perf_counter()
                Tb, tc, its = ctx.transmission_block(E_blk, kcols, block=blk, opts=om, return_cols=True)
                tb = time.perf_counter() - t0
                sb = ctx.last_stats()
                leg[f"block{blk}"] = {"solves_per_s": n / tb, "over_plain_mixed": tm / tb,
                                      "operator_applications_per_column": float(its.mean()),
                                      "columns_handed_to_plain_solver": int(sb["fp64_fallbacks"]),
                                      "max_rel_dT_vs_plain_mixed": float(np.max(np.abs(Tb - Tm) / np.abs(Tm)))}
        except B.RsnError as exc:
            leg["error"] = str(exc)
        result["block_T"] = leg

    # ---- many uneven junctions in one slot pool ----------------------------
    if rank == 0 and args.batch_junctions > 0:
        bj = P.batched_junctions()[: args.batch_junctions]
        bctx = [B.Context(local).set_junction(x) for x in bj]
        bE = [np.linspace(0.16, 0.24, args.batch_energies) for _ in bj]
        bcols = [x.right_columns()[:: args.batch_col_stride] for x in bj]
        ob = B.default_opts(B.RSN_MIXED, deadline_ms=args.deadline * 1e3)
        B.batch_transmission(bctx[:2], bE[:2], bcols[:2], ob)  # untimed warm-up (pool set-up, kernels loaded)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.batch_transmission(bctx, bE, bcols, ob)
        tb = time.perf_counter() - t0
        sb = bctx[0].last_stats()
        nb = sum(e.size * c.size for e, c in zip(bE, bcols))
        result["batched_junctions"] = {
            "sample": f"{len(bj)} seeded uneven junctions (cross-sections 12..32, 64..192 planes, CAP 6..10, "
                      f"5..30 wells), {args.batch_energies} energies in [0.16, 0.24] Ha each, every "
                      f"{args.batch_col_stride}th right-CAP column: {nb} forward solves in one slot pool, mixed "
                      "precision; host-timed library call",
            "columns_per_s": nb / tb, "seconds": tb, "krylov_iters_per_solve": sb["krylov_iters"] / nb,
            "fp64_fallbacks": sb["fp64_fallbacks"],
        }
        for x in bctx:
            x.close()

    # ---- parity against the oracle's golden columns ------------------------
    if rank == 0 and not args.no_fp64:
        gold = load_golden()
        if gold:
            rows = []
            for k, (E, gc, tg) in sorted(gold.items()):
                Tg = 4.0 * float(np.sum(j.gamma_r[gc] * tg))
                row = {"energy_index": k, "E": E, "T_oracle": Tg}
                for name, prec in (("fp64", B.RSN_FP64), ("mixed", B.RSN_MIXED)):
                    x, _, _ = ctx.solve_columns([E], gc, B.default_opts(prec))
                    xv = x[0]
                    gl = torch.tensor(j.gamma_l, device=xv.device)
                    tc = (gl[None, :] * (xv.real ** 2 + xv.imag ** 2)).sum(1).cpu().numpy()
                    T = float(ctx.transmission([E], gc, B.default_opts(prec))[0])
                    row[f"T_{name}"] = T
                    row[f"rel_dT_{name}"] = abs(T - Tg) / abs(Tg)
                    row[f"max_rel_dt_col_{name}"] = float(np.max(np.abs(tc - tg) / np.abs(tg)))
                rows.append(row)
            result["parity"] = {"golden": os.path.relpath(GOLDEN, ROOT), "columns": int(next(iter(gold.values()))[1].size),
                                "per_energy": rows}
    ctx.close()

    # ---- CPU oracle baseline (rank 0 at N = 1 only) ------------------------
    if rank == 0:
        if world == 1 and not args.no_cpu:
            cores = min(cpu_cores(), 16)
            Es = [energy_for(rank, world, k) for k in timed[:2]]
            pairs = sample_pairs(cols, Es, cores)
            v, wall_cpu = oracle_sample(pairs, cores)
            result["cpu_baseline"] = {
                "value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{len(pairs)} columns of the step's column set at the first two timed energies "
                          f"({', '.join(f'{e:.5f}' for e in Es)} Ha), one per core, each a forward and an adjoint "
                          f"solve by the oracle's Krylov route (complex128, certified true residual) to relative "
                          f"residual {CPU_SAMPLE_RTOL:g}; wall {wall_cpu:.1f} s",
            }
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    if rank != 0:
        return
    import numpy as np
    from paper_1401_0782_gb300 import problems as P
    j = P.molecular_junction(seed=1)
    cols = j.right_columns()
    if args.cols_per_step and args.cols_per_step < cols.size:
        cols = cols[:: int(np.ceil(cols.size / args.cols_per_step))]
    cores = min(cpu_cores(), 16)
    times = []
    for k in range(args.warmup + args.steps):
        pairs = sample_pairs(cols, [energy_for(0, 1, k)], cores)
        v, wall = oracle_sample(pairs, cores)
        if k >= args.warmup:
            times.append(wall)
    total = args.steps * cores
    value = total / sum(times)
    sample = (f"{cores} columns of the bench step's column set per step at that step's energy, one per core, "
              f"each a forward and an adjoint solve by the oracle's Krylov route (complex128, certified true "
              f"residual) to relative residual {CPU_SAMPLE_RTOL:g}")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("mixed precision (complex FP32 COCG + FP64 refinement to 1e-10)",
                                                "oracle (CPU, complex FP64)"), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cols-per-step", type=int, default=288,
                    help="columns per step: every k-th of the 4,608 right-CAP columns (0 = all)")
    ap.add_argument("--roofline-steps", type=int, default=2, help="steps of the event-timed roofline pass")
    ap.add_argument("--fwd-energies", type=int, default=6, help="energies of the forward-T comparison")
    ap.add_argument("--fwd-cols", type=int, default=1152,
                    help="columns of the forward-T comparison, every k-th of the 4,608 (0 = all)")
    ap.add_argument("--window-energies", type=int, default=16, help="energies of the shifted-COCG window leg (0 = skip)")
    ap.add_argument("--window-cols", type=int, default=128, help="columns of the shifted-COCG window leg")
    ap.add_argument("--block-cols", type=int, default=288, help="columns of the block-COCG leg (0 = skip)")
    ap.add_argument("--batch-junctions", type=int, default=64, help="junctions of the slot-pool leg (0 = skip)")
    ap.add_argument("--batch-energies", type=int, default=8, help="energies per junction in the slot-pool leg")
    ap.add_argument("--batch-col-stride", type=int, default=256, help="every k-th right-CAP column in the pool leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the forward-T, window and parity legs")
    ap.add_argument("--deadline", type=float, default=240.0, help="seconds allowed per library call")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
