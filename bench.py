"""Benchmark: vertex-steps/s of the DEC split-step march on one B300 (or N
independent replicas under torchrun), with the HBM roofline of the march
kernel, an end-to-end number through the host-buffer entry point, and the
CPU oracle as a reported baseline.

Workload (default): 16 step-index fibers of the paper's Table II (core radius
1, DEC disk of radius 4, V = -V#^2 in the cladding, Kerr ratio 2.2/2.8) with
20k..500k vertices, 16 launch fields each (seeded Hermite-Gauss
superpositions), dz = 5e-4, complex64 (FP32 arithmetic, FP64 diagnostics),
all advanced by one persistent launch per call.  A "step" is one z-step of
all 256 fields.  Its working set (~1.4 GB) is far larger than the 126 MB L2,
so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
METRIC = "vertex-steps/s (complex field) + % HBM roofline, FP32/batched vs plain FP64 on GPU"
UNIT = "vertex-steps/s"

# DRAM bytes (read + write) per algorithmic byte of the march kernels on this
# workload, per launch shape (the tile-staged kernel per ring slots and walk
# direction; the dataflow kernel per tile assignment, walk skip and walk
# direction), from an ncu capture of this bench's own launches (all of the
# autotuner's 3-step trial launches of these two kernels), valid for the
# kernel source whose hash is recorded with them; traffic is reported as
# null for another source, kernel or shape.
TRAFFIC_RATIO = {"march_tile_kernel:slots3:rev": 0.9351, "march_tile_kernel:slots2:rev": 0.9344,
                 "march_tile_kernel:slots3:fwd": 0.9879, "march_tile_kernel:slots2:fwd": 0.9875,
                 "march_flow_kernel:chunks:skip4:rev": 0.9624, "march_flow_kernel:chunks:skip8:rev": 0.9776,
                 "march_flow_kernel:chunks:skip16:rev": 0.9892, "march_flow_kernel:ranges:skip8:rev": 0.9835,
                 "march_flow_kernel:chunks:skip8:fwd": 0.9940, "march_flow_kernel:ranges:skip8:fwd": 0.9898}
TRAFFIC_SRC_HASH = "1bbcca780702978b"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("kernels.cuh", "api.cu"):
        with open(os.path.join(ROOT, "paper_2608_03587_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    try:
        with open(PEAKS_PATH) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        # nvidia-smi indexes physical GPUs: map through CUDA_VISIBLE_DEVICES
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ids = [v.strip() for v in vis.split(",")] if vis else []
        self.gpu = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "1", "yes"):
                        reasons.add(n)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workload
def build_workload(args, rank: int):
    from paper_2608_03587_b300 import workloads as W
    return W.batched_fibers(n_meshes=args.meshes, fields_per_mesh=args.fields, n_min=args.fiber_min,
                            ratio=args.fiber_ratio, seed=shard_seed(rank))


def traffic_shape_key(kernel_name, fused_kernel, cfg):
    """Key of TRAFFIC_RATIO for the launch shape a plan's config describes:
    the tile-staged kernel by ring slots and walk direction, the dataflow
    kernel by tile assignment, walk skip and walk direction."""
    walk = "fwd" if cfg.get("forward_walk") else "rev"
    if fused_kernel == 3:
        return "%s:%s:skip%d:%s" % (kernel_name, "ranges" if cfg.get("flow_ranges") else "chunks",
                                    cfg.get("flow_skip", 0), walk)
    if fused_kernel == 1:
        return "%s:slots%d:%s" % (kernel_name, cfg.get("tile_slots_used", 0), walk)
    return kernel_name


def algorithmic_bytes_per_step(mesh_infos, fields, degrees, scalar_bytes=8):
    """Bytes the degree-M Clenshaw chain must move per z-step (all meshes):
    per vertex-field, M * (S_op / B + 4 s) + 3 r / B with S_op = (4 + r) d + 4 + r
    (column index and weight per off-diagonal entry, diagonal, row pointer),
    s = 8 (complex64) or 16 (complex128), r = s / 2 the real size, and 3 r B of
    per-vertex epilogue data (v, chib, sigma): S_op = 8 d + 8, 12 B in FP32."""
    r = scalar_bytes / 2
    total = 0.0
    for info, B, M in zip(mesh_infos, fields, degrees):
        s_op = (4.0 + r) * info["mean_degree"] + 4.0 + r
        per_vf = M * (s_op / B + 4 * scalar_bytes) + 3.0 * r / B
        total += per_vf * info["n_vertices"] * B
    return total


def star0_rel_error(api, mesh, a, b):
    """*0-weighted relative L2 difference per field of two device fields
    [N0, B] (a against the reference b), from the library's FP64 diagnostics
    (power of the difference over power of the reference)."""
    import torch
    d = (a.to(torch.complex128) - b.to(torch.complex128)).contiguous()
    pd = api.diagnostics(mesh, d)["power"]
    pb = api.diagnostics(mesh, b.to(torch.complex128).contiguous())["power"]
    return np.sqrt(pd / pb)


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings (all ranks get the result)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def shard_seed(rank: int) -> int:
    """Replicas (weak scaling): every rank advances its own independent batch
    of the same shape; the launch-field seed differs per rank."""
    return 4 + 1000 * rank


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2608_03587_b300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t0 = time.time()
    wl = build_workload(args, rank)
    meshes = [api.Mesh.from_workload(m, p=wl.p) for m in wl.meshes]
    fields = [int(p.shape[1]) for p in wl.psi0]
    plan = api.Plan(meshes, fields, "c64")
    setup_s = time.time() - t0
    t_tune = time.time()
    tune = plan.autotune(wl.dz, trial_steps=3) if args.variant == "fused" else None
    tune_s = time.time() - t_tune
    psis = [torch.from_numpy(p).to(dev, torch.complex64).contiguous() for p in wl.psi0]
    infos = [m.info() for m in meshes]
    degrees = [plan.degree(i, wl.dz) for i in range(len(meshes))]
    units_per_step = sum(inf["n_vertices"] * B for inf, B in zip(infos, fields))

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up: W untimed steps (also captures the CUDA graph of this step count)
    plan.propagate(psis, wl.dz, args.warmup, variant=args.variant)
    plan.propagate(psis, wl.dz, args.steps, variant=args.variant)   # graph for K steps captured outside the timed region
    sync_all()
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        sync_all()
        ev0.record(stream)
        plan.propagate(psis, wl.dz, args.steps, variant=args.variant)
        ev1.record(stream)
        sync_all()
    ms = ev0.elapsed_time(ev1)
    march_ms = plan.last_march_ms()
    cfg = plan.config()
    clocks = clk.summary()

    # end to end through the host-buffer entry point (pinned host fields;
    # H2D of every field, the K-step march, D2H of every field and the diagnostics)
    host = [torch.from_numpy(p.astype(np.complex64)).pin_memory() for p in wl.psi0]
    plan.propagate_host(host, wl.dz, args.steps, variant=args.variant)
    sync_all()
    t_e2e = time.perf_counter()
    plan.propagate_host(host, wl.dz, args.steps, variant=args.variant)
    sync_all()
    e2e_s = time.perf_counter() - t_e2e
    io_bytes = sum(h.numel() * 8 for h in host)

    ms, march_ms, e2e_ms = max_over_ranks([ms, march_ms, e2e_s * 1e3], world, dev)

    alg_step = algorithmic_bytes_per_step(infos, fields, degrees)
    peak, peak_kind = hbm_peak()
    achieved = alg_step * args.steps / (march_ms * 1e-3) / 1e9
    value = units_per_step * args.steps * world / (ms * 1e-3)
    e2e_value = units_per_step * args.steps * world / (e2e_ms * 1e-3)
    # kernels of ours per timed call: permute in / out per mesh, the march
    # kernel, two diagnostic kernels per mesh
    launches = 1 + 4 * len(meshes)
    fk = cfg.get("fused_kernel", 0) if args.variant == "fused" else {"pairs": 2, "rows": 0, "flow": 3}.get(args.variant, 0)
    tiled = fk >= 1
    kernel_name = {3: "march_flow_kernel", 2: "march_pair_kernel", 1: "march_tile_kernel"}.get(
        fk, "march_kernel<float,%d>" % cfg["fields_padded"])
    traffic = None
    traffic_key = traffic_shape_key(kernel_name, fk, cfg)
    if traffic_key in TRAFFIC_RATIO and TRAFFIC_SRC_HASH == kernel_source_hash():
        traffic = TRAFFIC_RATIO[traffic_key] * alg_step * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": "batched step-index fibers: %d meshes (%d..%d vertices) x %d fields, dz=%g, c64"
                        % (len(meshes), min(i["n_vertices"] for i in infos), max(i["n_vertices"] for i in infos),
                           fields[0], wl.dz),
            "vertices_total": int(sum(i["n_vertices"] for i in infos)), "fields_per_mesh": fields[0],
            "cheb_degree_min": int(min(degrees)), "cheb_degree_max": int(max(degrees)),
            "ordering": "hilbert", "parallelism": "replicas" if world > 1 else "single",
            "grid": cfg["pair_grid"] if fk == 2 else cfg["flow_grid"] if fk == 3 else cfg["tile_grid"] if tiled else cfg["grid"],
            # the dataflow kernel has one warp more than the tile-staged kernel (its publisher)
            "block": cfg["tile_block"] + (32 if fk == 3 else 0) if tiled else cfg["block"],
            "passes_per_step": cfg["passes"] if fk == 2 else None,
            "march_kernel": kernel_name, "tile_slots": cfg["tile_slots_used"] if tiled else 0,
            "forward_walk": cfg["forward_walk"],
            "autotune": None if tune is None else {k: tune[k] for k in ("kernel", "ctas_per_sm", "tile_slots",
                                                                        "forward_walk", "walk_skip", "flow_ranges",
                                                                        "values_per_thread", "ms_per_step",
                                                                        "candidates")},
            "autotune_s": round(tune_s, 2),
            "cuda_graph": bool(cfg["graphs"]),
            "l2": "working set %.2f GB > 126 MB L2; no flush" % (units_per_step * 8 * 4 / 1e9),
            "setup_s": round(setup_s, 2),
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": kernel_name,
                     "kernel_ms": march_ms, "alg_bytes_per_launch": alg_step * args.steps},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes / args.steps,
                "d2h_bytes_per_step": io_bytes / args.steps},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_plain:
        line["fp32_vs_fp64"], line["fp64_fused"] = fp64_batch_comparison(wl, meshes, plan, fields, infos, api, torch,
                                                                         dev, args.steps)
        line["fp64_plain"] = plain_fp64_reference(wl, meshes, api, torch, dev)
        line["fp64_plain"]["fp32_batched_speedup"] = value / world / line["fp64_plain"]["value"]
        line["fp64_plain"]["fp32_batched_error_max"] = line["fp32_vs_fp64"]["max"]
        line["fp64_plain"]["fp64_fused_speedup"] = line["fp64_fused"]["value"] / line["fp64_plain"]["value"]
        line["rk45"] = rk45_comparison(wl, meshes, api, torch, dev, args.steps)
    if rank == 0 and not args.no_side:
        side = set(args.side_workloads.split(","))
        line["single_field"] = single_field_runs(api, torch, dev, args.side_steps, peak, side)
        if "adjoint" in side:
            line["adjoint"] = adjoint_run(api, torch, dev)
        if "pml" in side:
            line["pml"] = pml_run(api, torch, dev, peak)
        if "element" in side:
            line["element_kerr"] = element_kerr_run(plan, wl, torch, dev, args.steps, units_per_step, ms, args.variant)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, wl)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(wl, args.cpu_meshes, 16, n_steps=args.cpu_steps)
    return line


def fp64_batch_comparison(wl, meshes, plan32, fields, infos, api, torch, dev, steps):
    """The timed batch again from its launch fields, outside the timed region:
    K steps through the complex64 plan and through a complex128 plan of the
    same meshes (the fused FP64 path), the FP32 result's *0-weighted relative
    error against FP64 per field, and the FP64 plan's own rate and roofline."""
    plan64 = api.Plan(meshes, fields, "c128")
    a = [torch.from_numpy(p).to(dev, torch.complex128).contiguous() for p in wl.psi0]
    b = [torch.from_numpy(p).to(dev, torch.complex64).contiguous() for p in wl.psi0]
    plan32.propagate(b, wl.dz, steps)
    plan64.propagate([x.clone() for x in a], wl.dz, 3)
    plan64.propagate([x.clone() for x in a], wl.dz, steps)          # graph of this step count
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan64.propagate(a, wl.dz, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    march_ms = plan64.last_march_ms()
    errs = np.concatenate([star0_rel_error(api, m, x, y) for m, x, y in zip(meshes, b, a)])
    degrees = [plan64.degree(i, wl.dz) for i in range(len(meshes))]
    alg = algorithmic_bytes_per_step(infos, fields, degrees, scalar_bytes=16) * steps
    peak, _ = hbm_peak()
    units = sum(i["n_vertices"] * B for i, B in zip(infos, fields)) * steps
    err = {"max": float(errs.max()), "median": float(np.median(errs)), "fields": int(errs.size), "steps": steps,
           "norm": "*0-weighted relative L2 of the complex field, per field, FP32 plan vs FP64 plan"}
    fp64 = {"value": units / (ms * 1e-3), "unit": UNIT, "steps": steps, "march_ms": march_ms,
            "cheb_degree_max": int(max(degrees)), "kernel": "march_kernel<double,%d>" % plan64.config()["fields_padded"],
            "hbm_alg_frac": alg / (march_ms * 1e-3) / 1e9 / peak,
            "sample": "the whole batch, complex128, fused persistent launch"}
    plan64.close()
    return err, fp64


def single_field_runs(api, torch, dev, steps, peak, which=("disk", "vortex")):
    """The single-field workloads as the library runs them (fused FP32 path,
    one field), each with its error against the fused FP64 run of the same
    steps: the 200k-vertex graded disk (elliptic Gaussian, absorber) and the
    1M-vertex multimode guide (charge-1 vortex).  Both working sets fit in the
    126 MB L2, so the HBM fraction (algorithmic bytes at B = 1) is not a
    bandwidth claim here; it is reported with the working set."""
    from paper_2608_03587_b300 import workloads as W
    out = {}
    for key, name, make in (("disk", "gaussian_disk_200k", W.gaussian_disk),
                            ("vortex", "vortex_multimode_1M", W.vortex_multimode)):
        if key not in which:
            continue
        wl = make()
        m = wl.meshes[0]
        mesh = api.Mesh.from_workload(m, p=wl.p)
        info = mesh.info()
        res = {}
        for prec, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
            plan = api.Plan([mesh], [1], prec)
            tune = plan.autotune(wl.dz, trial_steps=5)
            psi = torch.from_numpy(wl.psi0[0]).to(dev, dt).contiguous()
            plan.propagate([psi.clone()], wl.dz, steps)                  # graph capture, warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.propagate([psi], wl.dz, steps)
            e1.record()
            torch.cuda.synchronize()
            M = plan.degree(0, wl.dz)
            res[prec] = (psi, e0.elapsed_time(e1), plan.last_march_ms(), M, tune, plan.config())
            plan.close()
        psi32, ms, march_ms, M, tune, cfg = res["c64"]
        alg = algorithmic_bytes_per_step([info], [1], [M]) * steps
        err = float(star0_rel_error(api, mesh, psi32, res["c128"][0])[0])
        n0 = info["n_vertices"]
        out[name] = {
            "vertices": n0, "steps": steps, "dz": wl.dz, "cheb_degree": M, "value": n0 * steps / (ms * 1e-3),
            "unit": UNIT, "march_ms": march_ms, "kernel": "march_kernel<float,1>" if not cfg["fused_kernel"]
            else "march_tile1_kernel", "autotune": {k: tune[k] for k in ("kernel", "ctas_per_sm", "forward_walk",
                                                                        "values_per_thread", "candidates")},
            "alg_bytes_per_vertex_step": alg / steps / n0, "hbm_alg_frac": alg / (march_ms * 1e-3) / 1e9 / peak,
            "working_set_mb": round((n0 * (8 * info["mean_degree"] + 8) + 4 * 8 * n0 + 12 * n0) / 1e6, 1),
            "fp32_vs_fp64": err, "fp64_value": n0 * steps / (res["c128"][1] * 1e-3),
            "fp64_cheb_degree": res["c128"][3]}
        mesh.close()
    return out


def element_kerr_run(plan, wl, torch, dev, steps, units_per_step, lumped_ms, variant):
    """The timed batch with the element-averaged Kerr term (Eq. 14: the phase
    from Q^T D Q of the intensities, one more neighbour pass per step after
    the last Clenshaw stage) instead of the lumped one: the same plan and
    launch shape, K steps from the launch fields (a CUDA graph replay, timed
    on its own after a capture call)."""
    psis = [torch.from_numpy(p).to(dev, torch.complex64).contiguous() for p in wl.psi0]
    plan.propagate(psis, wl.dz, steps, kerr="element", variant=variant)       # capture
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.propagate(psis, wl.dz, steps, kerr="element", variant=variant)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": units_per_step * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "march_ms": plan.last_march_ms(), "time_vs_lumped": ms / lumped_ms}


def pml_alg_bytes_per_vertex_field_step(M, mean_degree, B, real_bytes):
    """Bytes the march on the stretched operators must move per vertex-field
    and z-step: per stage the complex weights and columns of the row's SELL
    entries ((4 + 2 r) per entry, shared by the B fields) and four field
    accesses (g, psi and b_{k+2} read, the stage's output written, s = 2 r
    each); per step the diagonal flow's read and write of psi and its complex
    v, chib and real sigma (5 r per vertex)."""
    r = real_bytes
    s = 2 * r
    return M * ((4.0 + 2.0 * r) * mean_degree / B + 4.0 * s) + 2.0 * s + 5.0 * r / B


def pml_run(api, torch, dev, peak, steps=20):
    """The split-step march on the complex-stretched operators of a PML: a
    200k-vertex graded step-index fiber with the layer from r = 3 to 4
    (sigma_max 4, quadratic), 16 Hermite-Gauss superpositions, dz = 5e-4,
    complex64 and complex128, each through decbpm_propagate (persistent march
    or per-term launches, by the library's size rule), with the complex64
    fields' error against complex128 (*0-weighted, max over fields), the
    Chebyshev degree on the stretched spectrum and the whole call's rate as a
    fraction of the HBM roof (algorithmic bytes of the march; the working
    set, about 0.6 GB in complex64, exceeds L2)."""
    from paper_2608_03587_b300 import workloads as W
    coords, tris = W.mesh_disk_graded(4.0, 200000, 2.0, interfaces=(1.0,), seed=91, grade_from=1.0)
    V, chi = W.step_index_materials(coords, tris)
    mesh = api.Mesh(coords, tris, V, chi)
    api.set_pml(mesh, r_inner=3.0, r_outer=4.0, sigma_max=4.0, order=2)
    B, dz = 16, 5e-4
    psi0 = np.ascontiguousarray(W.hg_superpositions(coords, B, np.random.default_rng(91), power=4.0))
    n0 = coords.shape[0]
    info = mesh.info()
    out = {"vertices": int(n0), "fields": B, "steps": steps, "dz": dz}
    res = {}
    for prec, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
        psi = torch.from_numpy(psi0).to(dev, dt).contiguous()
        api.propagate(mesh, psi.clone(), dz, 2)                          # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.propagate(mesh, psi, dz, steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[prec] = psi
        M = api.pml_degree(mesh, dz, prec)
        alg = pml_alg_bytes_per_vertex_field_step(M, info["mean_degree"], B, 4 if prec == "c64" else 8) * n0 * B * steps
        out[prec] = {"value": n0 * B * steps / (ms * 1e-3), "unit": UNIT, "ms": ms, "cheb_degree": M,
                     "hbm_alg_frac": alg / (ms * 1e-3) / 1e9 / peak}
    out["fp32_vs_fp64"] = float(np.max(star0_rel_error(api, mesh, res["c64"], res["c128"])))
    out["fp32_speedup"] = out["c64"]["value"] / out["c128"]["value"]
    mesh.close()
    return out


def adjoint_run(api, torch, dev):
    """Cost of differentiation on the photonic-crystal-fiber workload (300k
    vertices, 60 holes, 2000 steps): the forward march and decbpm_adjoint
    (forward with sqrt(N) checkpoints, recomputation, backward march, FP64
    overlap objective) in vertex-steps/s of forward-equivalent work, FP32 and
    FP64."""
    from paper_2608_03587_b300 import workloads as W
    wl = W.pcf()
    m = wl.meshes[0]
    mesh = api.Mesh.from_workload(m, p=wl.p)
    n0, N = mesh.n_vertices, wl.n_steps
    out = {"vertices": n0, "steps": N, "checkpoints": int(math.ceil(math.sqrt(N)))}
    ref = None
    for prec, dt in (("c128", torch.complex128), ("c64", torch.complex64)):
        psi0 = torch.from_numpy(wl.psi0[0]).to(dev, dt).contiguous()
        fwd = psi0.clone()
        api.propagate(mesh, fwd.clone(), wl.dz, 3)
        torch.cuda.synchronize()
        t = time.perf_counter()
        api.propagate(mesh, fwd, wl.dz, N)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t
        if ref is None:
            # the target: the unperturbed guide's output, phase-shifted and mixed
            # with a narrower Gaussian, so that J is not at its maximum (where
            # dJ/dv would vanish by cancellation)
            ref = fwd.to(torch.complex128) * complex(math.cos(0.2), math.sin(0.2)) + 0.1 * torch.from_numpy(
                W.gaussian(m.coords, w=0.4)).to(dev, torch.complex128).reshape(fwd.shape)
        target = ref.to(dt).contiguous()
        t = time.perf_counter()
        J, gv, g0 = api.adjoint(mesh, psi0, target, wl.dz, N)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t
        out[prec] = {"forward_value": n0 * N / t_fwd, "adjoint_value": n0 * N / t_adj, "unit": UNIT,
                     "forward_s": t_fwd, "adjoint_s": t_adj, "adjoint_over_forward": t_adj / t_fwd, "J": float(J[0])}
        if prec == "c128":
            out["_gv64"] = gv
        else:
            gv64 = out.pop("_gv64")
            out["c64"]["grad_v_vs_fp64"] = float(torch.linalg.vector_norm(gv - gv64) / torch.linalg.vector_norm(gv64))
    mesh.close()
    return out


def rk45_comparison(wl, meshes, api, torch, dev, steps):
    """The paper's own integrator (adaptive Dormand-Prince, rtol 1e-9,
    atol 1e-11) on the GPU against the fused FP64 split-step march, both over
    z = steps * dz on the largest fiber, first field."""
    i = int(np.argmax([m.n_vertices for m in meshes]))
    psi0 = torch.from_numpy(np.ascontiguousarray(wl.psi0[i][:, 0])).to(dev, torch.complex128)
    z = steps * wl.dz
    a = psi0.clone()
    api.propagate(meshes[i], a, wl.dz, steps)
    a = psi0.clone()
    torch.cuda.synchronize()
    t = time.perf_counter()
    api.propagate(meshes[i], a, wl.dz, steps)
    torch.cuda.synchronize()
    split_ms = (time.perf_counter() - t) * 1e3
    b = psi0.clone()
    torch.cuda.synchronize()
    t = time.perf_counter()
    st = api.rk45(meshes[i], b, z, rtol=1e-9, atol=1e-11)
    torch.cuda.synchronize()
    rk_ms = (time.perf_counter() - t) * 1e3
    diff = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    return {"sample": "largest fiber (%d vertices), 1 field, c128, z=%g" % (meshes[i].n_vertices, z),
            "rk45_ms": rk_ms, "split_step_ms": split_ms, "split_step_speedup": rk_ms / split_ms,
            "rk45_accepted": int(st["n_accepted"]), "rk45_rejected": int(st["n_rejected"]),
            "rk45_rhs": int(st["n_rhs"]), "rel_l2_difference": diff}


def plain_fp64_reference(wl, meshes, api, torch, dev):
    """The plain single-field FP64 GPU path (unfused CSR SpMV + update
    launches per Chebyshev term) on the largest fiber, first field."""
    i = int(np.argmax([m.n_vertices for m in meshes]))
    psi = torch.from_numpy(np.ascontiguousarray(wl.psi0[i][:, 0])).to(dev, torch.complex128)
    api.propagate(meshes[i], psi, wl.dz, 1, variant="plain")
    torch.cuda.synchronize()
    n = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.propagate(meshes[i], psi, wl.dz, n, variant="plain")
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": meshes[i].n_vertices * n / (ms * 1e-3), "unit": UNIT, "steps": n,
            "sample": "largest fiber (%d vertices), 1 field, c128, %d steps" % (meshes[i].n_vertices, n)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(wl, n_meshes, n_steps):
    """Time the FP64 oracle (plain numpy/scipy) on the first field of the
    n_meshes smallest fibers for n_steps steps; returns (vertex-steps, seconds)."""
    from oracle import bpm, dec
    order = np.argsort([m.n_vertices for m in wl.meshes])[:n_meshes]
    units, secs = 0, 0.0
    for i in order:
        m = wl.meshes[i]
        ops = dec.Operators(m.coords, m.cells, m.V_cell, m.chi_cell)
        psi = wl.psi0[i][:, 0]
        t = time.perf_counter()
        bpm.propagate(ops, wl.p, psi, wl.dz, n_steps, m.sigma)
        secs += time.perf_counter() - t
        units += m.n_vertices * n_steps
    return units, secs


def cpu_baseline(args, wl):
    units, secs = oracle_sample(wl, args.cpu_meshes, args.cpu_steps)
    return {"value": units / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first field of the %d smallest fibers, %d steps each (%d vertex-steps, %.1f s); "
                      "numpy/scipy single thread" % (args.cpu_meshes, args.cpu_steps, units, secs)}


def _oracle_task(task):
    """One (mesh, field) oracle march in a worker process; returns
    (vertex-steps, seconds of the march alone, worker pid)."""
    coords, cells, V, chi, sigma, p, psi, dz, n_steps = task
    from oracle import bpm, dec
    ops = dec.Operators(coords, cells, V, chi)
    t = time.perf_counter()
    bpm.propagate(ops, p, psi, dz, n_steps, sigma)
    return coords.shape[0] * n_steps, time.perf_counter() - t, os.getpid()


def cpu_baseline_all_cores(wl, n_meshes, n_fields, cores=None, n_steps=1):
    """The oracle on every host core: independent (mesh, field) marches of the
    n_meshes smallest fibers (n_fields fields each, n_steps steps), one process per
    core (spawn start: the parent already holds a CUDA context), one thread
    per process.  Throughput = all vertex-steps / the largest per-process march
    time (process start-up and assembly excluded, as the GPU's setup is)."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    order = np.argsort([m.n_vertices for m in wl.meshes])[:n_meshes]
    tasks = []
    for i in order:
        m = wl.meshes[i]
        for b in range(min(n_fields, wl.psi0[i].shape[1])):
            tasks.append((m.coords, m.cells, m.V_cell, m.chi_cell, m.sigma, wl.p, wl.psi0[i][:, b], wl.dz, n_steps))
    workers = max(1, min(cores, len(tasks)))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    busy = {}
    units = 0
    with mp.get_context("spawn").Pool(workers) as pool:
        for u, sec, pid in pool.imap_unordered(_oracle_task, tasks, chunksize=1):
            units += u
            busy[pid] = busy.get(pid, 0.0) + sec
    wall = max(busy.values())
    return {"value": units / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": "%d fields x %d steps on the %d smallest fibers (%d vertex-steps), one process per core, "
                      "slowest process %.1f s" % (len(tasks), n_steps, n_meshes, units, wall)}


def run_reference(args, rank, world):
    """Reference arm: the CPU FP64 oracle, timed as it stands on the host."""
    if rank != 0:
        return None
    wl = build_workload(args, 0)
    per_step = []
    tot_units, tot_s = 0, 0.0
    for k in range(args.warmup + args.steps):
        units, secs = oracle_sample(wl, args.ref_meshes, 1)
        if k >= args.warmup:
            per_step.append(secs)
            tot_units += units
            tot_s += secs
    value = tot_units / tot_s
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched step-index fibers (bounded sample: first field of the %d smallest "
                               "fibers per step)" % args.ref_meshes},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "first field of the %d smallest fibers, 1 z-step per timed step"
                                   % args.ref_meshes},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--meshes", type=int, default=16)
    ap.add_argument("--fields", type=int, default=16)
    ap.add_argument("--fiber-min", type=int, default=20_000, help="vertices of the smallest fiber")
    ap.add_argument("--fiber-ratio", type=float, default=25.0, help="largest / smallest fiber size")
    ap.add_argument("--cpu-meshes", type=int, default=8)
    ap.add_argument("--cpu-steps", type=int, default=3, help="oracle steps per field of the CPU baselines")
    ap.add_argument("--ref-meshes", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the single-field and adjoint side runs")
    ap.add_argument("--side-steps", type=int, default=200, help="steps of the single-field side runs")
    ap.add_argument("--side-workloads", default="disk,vortex,adjoint,pml,element",
                    help="side runs to make: any of disk (200k single field), vortex (1M), adjoint (300k PCF), "
                         "pml (200k fiber with a PML, 16 fields), element (the batch with element-averaged Kerr)")
    ap.add_argument("--variant", choices=["fused", "rows", "pairs", "flow"], default="fused",
                    help="fused: the autotuner's choice; pairs: the stage-pair kernel; rows: the row kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
