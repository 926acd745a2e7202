"""Benchmark: H' build throughput (GB/s of algorithmic bytes) on GB300.

One step = H -> H' over every depth of the workload (all steps of the map:
per-depth split, index map, flip, exchange, data movement), with the input
resident in HBM.  The headline form is the batched launch (one CUDA graph in
the autotuner's form: persistent CTAs, one tile per CTA, or per-depth grids); the
plain per-depth form is timed beside it on the same GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload highres|mid|ragged|autograd|tiny] [--dtype f32|f16]

Algorithmic bytes per step = 2 * sum_z Nx*Ny*Ks_z*Kt_z * esize (every element
read once and written once).  Inputs are larger than L2 (129 MB) for the
default workload, so no flush runs between steps.  Under torchrun every
rank maps its own copy of the workload (independent problems, no
collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H' build GB/s and % of HBM peak on 1 GB300, batched vs per-depth form, bit-exact"
SPEC_GBS = 8000.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_sha():
    """Hash of the gather kernels' source: lfbp_device.cuh, the consumer
    headers it includes, and the device part of lfbp.cu (everything before its
    host section)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2003_09133_gb300", "csrc")
    for name in ("lfbp_device.cuh", "lfbp_stripes.cuh", "lfbp_pairs.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "lfbp.cu"), "rb") as fh:
        h.update(fh.read().split(b"// ====================================================================== host")[0])
    return h.hexdigest()[:16]


def _traffic_record(workload, dtype, kernel):
    """DRAM bytes per step from a committed ncu summary of `kernel`, if the
    kernels' source is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        for ent in rec.values():
            if (ent.get("workload") == workload and ent.get("dtype") == dtype and
                    ent.get("kernel") == kernel and ent.get("source_sha") == _kernel_source_sha()):
                return ent
    except Exception:
        pass
    return None


# the kernel that does the work of each batched form (lfbp_tune_batched's fifth value)
FORM_KERNEL = {0: "k_gather_persistent", 1: "k_gather_tiles", 2: "k_gather_depth"}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_ms=50):
        self.index, self.period_ms = index, period_ms
        self.proc, self.path = None, None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for _, _, flags in rows:
            for n, f in zip(names, flags[1:]):
                if f.lower() in ("active", "0x1", "1"):
                    seen.add(n)
        mhz = sorted(r[0] for r in rows)
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(seen)}


def _workload_desc(specs, dtype_override):
    if len(specs) == 1:
        s = specs[0]
        return (f"{s.name}: Nx=Ny={s.Nx}, Nz={s.Nz}, K_z {min(s.Ks)}..{max(s.Ks)} px, "
                f"ragged in depth, {dtype_override or s.dtype}")
    return f"{specs[0].name[:6]}: {len(specs)} arrays, mixed fp32/fp16, ragged"


def _dist():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world):
    """Largest value of x over all ranks (the step time every rank waits for)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_specs(specs, rank):
    """Rank r maps its own problem: same shapes, amplitude seeds offset by 1000*r."""
    import dataclasses
    if rank == 0:
        return specs
    return [dataclasses.replace(s, seed=s.seed + 1000 * rank) for s in specs]


def aggregate_gbs(step_bytes_per_rank, max_ms, world):
    """Whole-job GB/s: the bytes all ranks moved over the slowest rank's time."""
    return world * step_bytes_per_rank / (max_ms * 1e-3) / 1e9


def _cpu_oracle_rate(specs, Hs_host, dtype_override, budget_s=12.0, max_passes=32):
    """Time the CPU oracle (as it stands) on the workload: GB/s of algorithmic bytes."""
    import numpy as np
    import oracle
    done_bytes, t_total, passes = 0, 0.0, 0
    cores = oracle.threads(0)
    sample_desc = []
    while passes < max_passes and t_total < budget_s:
        for s, H in zip(specs, Hs_host):
            t0 = time.perf_counter()
            oracle.transpose(H, s.Nx, s.Ny, s.Ks, s.Kt)
            t_total += time.perf_counter() - t0
            done_bytes += 2 * H.nbytes
            if passes == 0:
                sample_desc.append(s.name)
            if t_total >= budget_s:
                break
        passes += 1
    # the same oracle on one thread, on the first array's middle depth (a few seconds)
    s, H = specs[0], Hs_host[0]
    import lfgen
    off = lfgen.depth_offsets(s)
    z = s.Nz // 2
    Hz = np.ascontiguousarray(H[off[z]:off[z + 1]])
    oracle.threads(1)
    t0 = time.perf_counter()
    oracle.transpose(Hz, s.Nx, s.Ny, [s.Ks[z]], [s.Kt[z]])
    t1 = time.perf_counter() - t0
    oracle.threads(cores)
    return {"value": done_bytes / t_total / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "seconds": round(t_total, 3),
            "sample": f"{done_bytes / 2 / 1e9:.2f} GB of H mapped by oracle.transpose "
                      f"({passes} pass(es) over {'+'.join(sample_desc)}; C, OpenMP {cores} threads)",
            "single_thread_GBps": round(2 * Hz.nbytes / t1 / 1e9, 3),
            "single_thread_sample": f"depth {z} of {s.name} (K = {s.Ks[z]}), 1 thread",
            "closed_form": _cpu_closed_form_rate(specs, Hs_host)}


def _cpu_closed_form_rate(specs, Hs_host, budget_s=6.0, max_passes=8):
    """The paper's method on the host cores: the closed-form rearrangement of
    Sec. 4 in C with OpenMP (oracle/lfbp_cpu_rearrange.c), over the whole
    workload on all cores, and on one depth on one core."""
    import numpy as np
    import oracle
    import lfgen
    cores = oracle.cpu_rearrange_threads(0)
    done, t_total, passes = 0, 0.0, 0
    while passes < max_passes and t_total < budget_s:
        for s, H in zip(specs, Hs_host):
            t0 = time.perf_counter()
            oracle.cpu_rearrange(H, s.Nx, s.Ny, s.Ks, s.Kt)
            t_total += time.perf_counter() - t0
            done += 2 * H.nbytes
        passes += 1
    s, H = specs[0], Hs_host[0]
    off = lfgen.depth_offsets(s)
    z = s.Nz // 2
    Hz = np.ascontiguousarray(H[off[z]:off[z + 1]])
    t0 = time.perf_counter()
    oracle.cpu_rearrange(Hz, s.Nx, s.Ny, [s.Ks[z]], [s.Kt[z]], 1)
    t1 = time.perf_counter() - t0
    oracle.cpu_rearrange_threads(cores)
    return {"value": round(done / t_total / 1e9, 3), "unit": "GB/s", "cores": cores,
            "kind": "the paper's closed-form rearrangement (Sec. 4), C with OpenMP",
            "sample": f"{passes} pass(es) over the whole workload ({done / 2 / 1e9:.2f} GB of H)",
            "single_thread_GBps": round(2 * Hz.nbytes / t1 / 1e9, 3),
            "single_thread_sample": f"depth {z} of {s.name} (K = {s.Ks[z]}), 1 thread"}


def _reference_sample(specs, budget_elems=48_000_000):
    """Evenly spaced depths of the workload holding about budget_elems elements."""
    import lfgen
    depths = []
    for ai, s in enumerate(specs):
        off = lfgen.depth_offsets(s)
        for z in range(s.Nz):
            depths.append((ai, z, off[z], s.Nx * s.Ny * s.Ks[z] * s.Kt[z]))
    total = sum(d[3] for d in depths)
    m = max(1, round(len(depths) * budget_elems / max(1, total)))
    stride = max(1, len(depths) // m)
    picks, acc = [], 0
    for d in depths[stride // 2::stride]:
        if picks and acc + d[3] > 1.5 * budget_elems:
            continue
        picks.append(d)
        acc += d[3]
    return picks, acc


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores, same metric and workload.

    Each step maps a fixed sample of the workload's depths (every k-th depth,
    about 48 M elements) with oracle.transpose, so that a run of --steps K
    stays within a few minutes; the value is that sample's GB/s.
    """
    import torch
    import lfgen
    import oracle
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    specs = _pick_specs(args)
    picks, acc = _reference_sample(specs)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    arrays = {}
    for ai in sorted({p[0] for p in picks}):
        s = specs[ai]
        arrays[ai] = lfgen.generate(s, device=dev).to(_torch_dtype(args, s)).cpu().numpy()
    sample = [(specs[ai], arrays[ai][off:off + n].copy(), z) for ai, z, off, n in picks]
    nbytes = sum(2 * h.nbytes for _, h, _ in sample)

    def one_step():
        for s, h, z in sample:
            oracle.transpose(h, s.Nx, s.Ny, [s.Ks[z]], [s.Kt[z]])

    for _ in range(args.warmup):
        one_step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one_step()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = nbytes / t / 1e9
    cores = oracle.threads(0)
    desc = (f"{len(sample)} of the workload's depths (evenly spaced), "
            f"{acc / 1e6:.1f} M elements, {nbytes / 2 / 1e9:.3f} GB of H) per step, "
            f"oracle.transpose in C with OpenMP")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype_name(args, specs), "data": "synthetic",
        "config": _config(args, specs),
        "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _torch_dtype(args, spec):
    import torch
    if args.dtype == "f16":
        return torch.float16
    if args.dtype == "f32":
        return torch.float32
    return spec.torch_dtype


def _dtype_name(args, specs):
    if args.dtype:
        return args.dtype
    names = sorted({s.dtype for s in specs})
    return "+".join(names)


def _pick_specs(args):
    import dataclasses
    import lfgen
    specs = lfgen.config_specs(args.workload)
    if args.depth_stride > 1:
        # every k-th depth only: a smaller case of the same shapes (for profiling)
        out = []
        for s in specs:
            keep = list(range(0, s.Nz, args.depth_stride))
            out.append(dataclasses.replace(
                s, Ks=tuple(s.Ks[z] for z in keep), Kt=tuple(s.Kt[z] for z in keep),
                radius=tuple(s.radius[z] for z in keep), name=s.name + f"/every{args.depth_stride}"))
        specs = out
    return specs


def _config(args, specs, world=1):
    import lfgen
    elems = sum(lfgen.array_elems(s) for s in specs)
    cfg = {"workload": _workload_desc(specs, args.dtype), "arrays": len(specs),
           "elements_per_rank": elems, "form": "batched (1 CUDA graph launch; the autotuner's form)",
           "l2": "inputs larger than L2 (no flush)" if elems * 2 > 129e6 else
                 "L2 flushed between steps"}
    if args.scaling == "strong":
        cfg["elements_per_rank"] = None
        cfg["elements_per_job"] = elems
        cfg["parallelism"] = f"depths split across {world} rank(s) (lfbp_plan_partition)"
    else:
        cfg["parallelism"] = f"{world} independent array(s), one per rank"
    return cfg


def run_ours(args):
    import numpy as np
    import torch
    import lfgen
    import paper_2003_09133_gb300 as lf

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    lf.load()
    strong = args.scaling == "strong"
    # weak: every rank maps its own array (seeds offset per rank); strong: the
    # ranks split the depths of one array (lfbp_plan_partition) and map their part
    specs = _pick_specs(args) if strong else rank_specs(_pick_specs(args), rank)
    plans, Hs, outs = [], [], []
    job_bytes = 0
    for s in specs:
        dt = _torch_dtype(args, s)
        full = lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, dt)
        H = lfgen.generate(s, device="cuda").to(dt)
        job_bytes += 2 * H.numel() * H.element_size()
        if strong:
            z0, z1 = full.partition(world, rank)
            if z1 <= z0:
                continue
            plans.append(full.sub_plan(z0, z1))
            Hs.append(H[full.depth_offset(z0):full.depth_offset(z1)].clone())  # 16-byte aligned
            del H
        else:
            plans.append(full)
            Hs.append(H)
        outs.append(torch.empty_like(Hs[-1]))
    torch.cuda.synchronize()
    step_bytes = sum(2 * h.numel() * h.element_size() for h in Hs)
    step_elems = sum(h.numel() for h in Hs)
    # whole-job bytes per step: every rank's own array (weak) or the one shared array (strong)
    job_total = job_bytes if strong else world * step_bytes
    flush = None
    if step_bytes < 2 * 129e6:
        flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step_batched():
        lf.backproject_batched(plans, Hs, outs)

    def step_plain():
        for p, h, o in zip(plans, Hs, outs):
            lf.backproject_array(p, h, o)

    step_ms = []  # the per-step times of the last timed() call (this rank)

    def timed(fn, steps, warmup, clocks=False):
        for _ in range(warmup):
            fn()
        lf.sync_status()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        _barrier(world)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        for a, b in ev:
            if flush is not None:
                flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        _barrier(world)
        if sampler:
            sampler.__exit__(None, None, None)
        lf.sync_status()
        ms = [a.elapsed_time(b) for a, b in ev]
        step_ms[:] = ms
        mean = sum(ms) / len(ms)
        return _max_over_ranks(mean, world), min(ms), (sampler.summary() if sampler else None)

    # launch shape of the batched form picked by the library's autotuner
    # (outside the timed region; later calls with these plans reuse it)
    tuned = None if args.no_tune else lf.tune_batched(plans, Hs, outs)
    t_batched, best_batched, clocks = timed(step_batched, args.steps, args.warmup, clocks=True)
    t_plain, best_plain, _ = timed(step_plain, max(3, args.steps // 4), max(3, args.warmup))

    # end to end through the C-ABI with host buffers: pinned host H -> device ->
    # H' -> pinned host, the copies of one chunk of depths overlapping the map
    # of the previous chunk (lfbp_backproject_array_host)
    e2e = None
    if not args.no_e2e:
        hosts = [h.cpu().pin_memory() for h in Hs]
        host_out = [torch.empty_like(h, device="cpu").pin_memory() for h in Hs]
        dev_in = [torch.empty_like(h) for h in Hs]

        def step_e2e():
            for p, hi, ho, di, do in zip(plans, hosts, host_out, dev_in, outs):
                lf.backproject_array_host(p, hi, ho, work=(di, do))

        n_e2e = max(3, min(args.steps, 20))
        t_e2e, best_e2e, _ = timed(step_e2e, n_e2e, 2)
        e2e_ms = sorted(step_ms)
        nbytes = sum(h.numel() * h.element_size() for h in Hs)

        # the host link alone: the same bytes copied host -> device
        # and device -> host at the same time on two streams, no map (context
        # for the e2e number: its floor)
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def link_only():
            cur = torch.cuda.current_stream()
            s_in.wait_stream(cur)
            s_out.wait_stream(cur)
            for hi, ho, di, do in zip(hosts, host_out, dev_in, outs):
                with torch.cuda.stream(s_in):
                    di.copy_(hi, non_blocking=True)
                with torch.cuda.stream(s_out):
                    ho.copy_(do, non_blocking=True)
            cur.wait_stream(s_in)
            cur.wait_stream(s_out)

        t_link, _, _ = timed(link_only, max(3, n_e2e // 4), 2)
        e2e = {"value": round(job_total / (t_e2e * 1e-3) / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": round(t_e2e, 3),
               # the spread of the steps behind the mean (this rank): sporadic
               # slow steps on a shared host show as a mean above the median
               "step_ms_median": round(e2e_ms[len(e2e_ms) // 2], 3),
               "step_ms_min": round(best_e2e, 3),
               "link_only_ms": round(t_link, 3),
               "link_only": "the same bytes copied both ways at once, no map (not timed in e2e)"}
        del hosts, host_out, dev_in

    peak, peak_kind = _peaks()
    achieved = step_bytes / (t_batched * 1e-3) / 1e9
    value = job_total / (t_batched * 1e-3) / 1e9
    kernel = FORM_KERNEL[tuned[4] if tuned else 1]
    traffic = None if strong else _traffic_record(args.workload, _dtype_name(args, specs), kernel)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_batched, 4),
        "higher_is_better": True, "scaling": args.scaling, "vs_baseline": None,
        "dtype": _dtype_name(args, specs), "data": "synthetic",
        "config": _config(args, specs, world),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": kernel,
                     "traffic": traffic["bytes_per_launch"] if traffic else None,
                     "algorithmic_bytes_per_launch": step_bytes},
        "pct_of_8TBps_spec": round(100 * achieved / SPEC_GBS, 2),
        "launch_shape": _tuned_desc(tuned) or "default (one tile per CTA, 64 KB tiles)",
        "elements_per_s": round(job_total * step_elems / step_bytes / (t_batched * 1e-3), 1)
        if step_bytes else 0.0,
        "best_ms_per_step": round(best_batched, 4),
        "plain": {"ms_per_step": round(t_plain, 4),
                  "value": round(job_total / (t_plain * 1e-3) / 1e9, 3),
                  "best_ms_per_step": round(best_plain, 4),
                  "launches_per_step": sum(p.Nz for p in plans), "kernel": "k_gather_depth"},
        "e2e": e2e,
        # kernel launches of the timed steps: one per step, or one grid per depth
        # of every array in the per-depth graph form
        "gpu_launches": (args.steps * (sum(p.Nz for p in plans) if (tuned and tuned[4] == 2) else 1)
                         if plans else 0),
        "clocks": clocks,
    }
    if not args.no_extra and not strong and args.workload == "highres" and args.dtype in (None, "f32"):
        line["extra"] = _extra_forms(lf, plans, specs, Hs, outs, timed, args, world)
    if rank == 0 and not args.no_cpu_baseline:
        Hh = [h.cpu().numpy() for h in Hs]
        line["cpu_baseline"] = _cpu_oracle_rate(specs, Hh, args.dtype)
    line["summary"] = _summary(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _summary(line):
    """The forms side by side in GB/s (batched / plain), last on the line."""
    out = {"headline": {"batched": line["value"], "plain": line["plain"]["value"],
                        "frac_of_measured_hbm": line["roofline"]["frac"]}}
    ex = line.get("extra") or {}
    for key in ("highres_fp16", "ragged", "mid", "highres_dense"):
        if key in ex:
            out[key] = {"batched": ex[key]["batched_GBps"], "plain": ex[key]["plain_GBps"]}
    ek = (ex.get("paper_window") or {}).get("even_K")
    if ek:
        out["even_K"] = {"batched": ek.get("batched_GBps"), "plain": ek.get("plain_GBps")}
    cb = line.get("cpu_baseline")
    if cb:
        out["cpu_GBps"] = {"oracle": round(cb["value"], 2), "cores": cb["cores"],
                           "closed_form": cb["closed_form"]["value"],
                           "closed_form_1_core": cb["closed_form"]["single_thread_GBps"]}
    return out


def _mid_extra(lf, timed, steps, world, no_tune=False):
    """The mid-resolution array (N = 15, 51 depths, K 45..165, fp32): the plain
    form (one launch per depth) beside the batched form."""
    import torch
    import lfgen
    s = lfgen.config_specs("mid")[0]
    plan = lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, torch.float32)
    H = lfgen.generate(s, device="cuda")
    O = torch.empty_like(H)
    nb = 2 * H.numel() * 4
    tuned = None if no_tune else lf.tune_batched([plan], [H], [O])
    tb, _, _ = timed(lambda: lf.backproject_batched([plan], [H], [O]), steps, 3)
    tp, _, _ = timed(lambda: lf.backproject_array(plan, H, O), steps, 3)
    res = {"workload": "mid: N=15, 51 depths, K_z 45..165, fp32", "bytes_per_step": nb,
           "batched_GBps": round(world * nb / (tb * 1e-3) / 1e9, 1),
           "plain_GBps": round(world * nb / (tp * 1e-3) / 1e9, 1),
           "batched_ms": round(tb, 4), "plain_ms": round(tp, 4), "plain_launches_per_step": s.Nz,
           "tuned": _tuned_desc(tuned)}
    del H, O
    torch.cuda.empty_cache()
    return res


def _extra_forms(lf, plans, specs, Hs, outs, timed, args, world):
    """The fp16-stored copy of the same array, and the ragged 16-array batch:
    batched persistent form next to the plain per-depth form."""
    import torch
    import lfgen
    res = {}
    steps = max(3, args.steps // 4)
    # fp16 storage of the same values (round to nearest even)
    p16 = [lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, torch.float16) for s in specs]
    h16 = [h.half() for h in Hs]
    o16 = [torch.empty_like(h) for h in h16]
    nb = sum(2 * h.numel() * 2 for h in h16)
    tuned16 = None if args.no_tune else lf.tune_batched(p16, h16, o16)
    tb, _, _ = timed(lambda: lf.backproject_batched(p16, h16, o16), steps, 3)
    tp, _, _ = timed(lambda: [lf.backproject_array(p, h, o) for p, h, o in zip(p16, h16, o16)],
                     steps, 3)
    res["highres_fp16"] = {"batched_GBps": round(world * nb / (tb * 1e-3) / 1e9, 1),
                           "plain_GBps": round(world * nb / (tp * 1e-3) / 1e9, 1),
                           "batched_ms": round(tb, 4), "plain_ms": round(tp, 4),
                           "tuned": _tuned_desc(tuned16)}
    del h16, o16
    torch.cuda.empty_cache()
    # the same array padded centrally to K = K_max at every depth (the dense
    # form of the workload; centred cropping commutes with the map)
    if len(specs) == 1:
        s = specs[0]
        Km = max(s.Ks)
        H = Hs[0]
        dplan = lf.Plan(s.Nx, s.Ny, [Km] * s.Nz, [Km] * s.Nz, torch.float32)
        Hd = torch.zeros(dplan.elems, dtype=torch.float32, device="cuda")
        for z in range(s.Nz):
            k, o = s.Ks[z], (Km - s.Ks[z]) // 2
            src = H[plans[0].depth_offset(z):plans[0].depth_offset(z + 1)].view(s.Nx, s.Ny, k, k)
            dst = Hd[dplan.depth_offset(z):dplan.depth_offset(z + 1)].view(s.Nx, s.Ny, Km, Km)
            dst[:, :, o:o + k, o:o + k] = src
        Od = torch.empty_like(Hd)
        nbd = 2 * Hd.numel() * 4
        dtuned = None if args.no_tune else lf.tune_batched([dplan], [Hd], [Od])
        tb, _, _ = timed(lambda: lf.backproject_batched([dplan], [Hd], [Od]), steps, 3)
        tp, _, _ = timed(lambda: lf.backproject_array(dplan, Hd, Od), steps, 3)
        res["highres_dense"] = {"K": Km, "bytes_per_step": nbd,
                                "batched_GBps": round(world * nbd / (tb * 1e-3) / 1e9, 1),
                                "plain_GBps": round(world * nbd / (tp * 1e-3) / 1e9, 1),
                                "batched_ms": round(tb, 4), "plain_ms": round(tp, 4),
                                "tuned": _tuned_desc(dtuned)}
        del Hd, Od
        torch.cuda.empty_cache()
    # the ragged batch: 16 arrays, mixed fp32 / fp16, one persistent launch
    rspecs = lfgen.config_specs("ragged")
    rplans = [lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, s.torch_dtype) for s in rspecs]
    rH = [lfgen.generate(s, device="cuda") for s in rspecs]
    rO = [torch.empty_like(h) for h in rH]
    nb = sum(2 * h.numel() * h.element_size() for h in rH)
    rtuned = None if args.no_tune else lf.tune_batched(rplans, rH, rO)
    tb, _, _ = timed(lambda: lf.backproject_batched(rplans, rH, rO), steps, 3)
    tp, _, _ = timed(lambda: [lf.backproject_array(p, h, o) for p, h, o in zip(rplans, rH, rO)],
                     steps, 3)
    res["ragged"] = {"arrays": len(rspecs), "bytes_per_step": nb,
                     "batched_GBps": round(world * nb / (tb * 1e-3) / 1e9, 1),
                     "plain_GBps": round(world * nb / (tp * 1e-3) / 1e9, 1),
                     "batched_ms": round(tb, 4), "plain_ms": round(tp, 4),
                     "plain_launches_per_step": sum(s.Nz for s in rspecs),
                     "tuned": _tuned_desc(rtuned)}
    del rH, rO
    torch.cuda.empty_cache()
    res["mid"] = _mid_extra(lf, timed, steps, world, args.no_tune)
    res["paper_window"] = _paper_window_extra(lf, specs, Hs, outs, timed, steps, world, args.no_tune)
    res["table1"] = _table1_extra(lf, world, args.no_tune)
    res["rl_step"] = _rl_extra(lf, timed, steps)
    res["autograd_step"] = _autograd_extra(lf, timed, steps)
    return res


def _paper_window_extra(lf, specs, Hs, outs, timed, steps, world, no_tune=False):
    """The headline array in the literal Eqs. (4)-(9) mode (entries the paper's
    loop ranges leave unwritten are zero-filled), batched and plain."""
    import torch
    pw = [lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, torch.float32, mode=lf.MAP_PAPER_WINDOW) for s in specs]
    nb = sum(2 * h.numel() * h.element_size() for h in Hs)
    tuned = None if no_tune else lf.tune_batched(pw, Hs, outs)
    tb, _, _ = timed(lambda: lf.backproject_batched(pw, Hs, outs), steps, 3)
    tp, _, _ = timed(lambda: [lf.backproject_array(p, h, o) for p, h, o in zip(pw, Hs, outs)],
                     steps, 3)
    res = {"mode": "MAP_PAPER_WINDOW", "batched_GBps": round(world * nb / (tb * 1e-3) / 1e9, 1),
           "plain_GBps": round(world * nb / (tp * 1e-3) / 1e9, 1),
           "batched_ms": round(tb, 4), "plain_ms": round(tp, 4), "tuned": _tuned_desc(tuned)}
    # even cut-outs (the literal Eq. 8): the same depths with every K one larger,
    # through the same tiled gather (the cropped odd cut-out under the window)
    if len(specs) == 1:
        s = specs[0]
        ke, kte = [k + 1 for k in s.Ks], [k + 1 for k in s.Kt]
        pe = lf.Plan(s.Nx, s.Ny, ke, kte, torch.float32, mode=lf.MAP_PAPER_WINDOW)
        He = torch.empty(pe.elems, dtype=torch.float32, device="cuda").uniform_()
        Oe = torch.empty_like(He)
        tuned_e = None if no_tune else lf.tune_batched([pe], [He], [Oe])
        tbe, _, _ = timed(lambda: lf.backproject_batched([pe], [He], [Oe]), steps, 3)
        te, _, _ = timed(lambda: lf.backproject_array(pe, He, Oe), steps, 3)
        nbe = 2 * pe.elems * 4
        res["even_K"] = {"K": "every highres K + 1", "bytes_per_step": nbe,
                         "batched_GBps": round(world * nbe / (tbe * 1e-3) / 1e9, 1),
                         "plain_GBps": round(world * nbe / (te * 1e-3) / 1e9, 1),
                         "batched_ms": round(tbe, 4), "plain_ms": round(te, 4),
                         "tuned": _tuned_desc(tuned_e),
                         "kernel": "k_gather_persistent / k_gather_depth (masked chunk path)"}
        del He, Oe
        torch.cuda.empty_cache()
    return res


# Table 1 of the paper: n_s = n_t, n_x, n_y and the paper's own time in seconds
# (MATLAB 2019a on an i7-6700K, precision not stated; context only), n_z = 11.
TABLE1 = [(89, 11, 11, 0.10), (177, 11, 11, 0.36), (287, 11, 11, 1.05), (507, 11, 11, 3.13),
          (91, 15, 15, 0.13), (121, 15, 15, 0.23), (211, 21, 21, 1.08), (249, 31, 31, 2.85),
          (311, 31, 31, 4.74), (307, 51, 51, 11.3), (181, 95, 55, 5.9)]


def _table1_extra(lf, world, no_tune=False, reps=5, rows=None, nz=11):
    """Every PSF-array size of Table 1 (11 depths of one K; K not a multiple of
    N; the last row the non-square 95 x 55 cell), fp32, seeded uniform values:
    one batched launch per array, in the launch shape the library's autotuner
    picks for it (`tuned`; the default shape's time beside it).  Inputs of
    0.04-10.8 GB per direction; arrays below 2 x L2 are timed with an L2 flush
    between launches."""
    import torch
    table = [t for t in TABLE1 if rows is None or t[0] in rows]
    nmax = max(nx * ny * k * k * nz for k, nx, ny, _ in table)
    gen = torch.Generator(device="cuda").manual_seed(7)
    Hbuf = torch.empty(nmax, dtype=torch.float32, device="cuda").uniform_(generator=gen)
    Obuf = torch.empty_like(Hbuf)
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device="cuda")
    out_rows = []
    for k, nx, ny, paper_s in table:
        plan = lf.Plan(nx, ny, [k] * nz, [k] * nz, torch.float32)
        H, O = Hbuf[:plan.elems], Obuf[:plan.elems]
        nb = 2 * plan.elems * 4

        def time_it():
            for _ in range(3):
                lf.backproject_batched([plan], [H], [O])
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            for a, b in ev:
                if nb < 2 * 129e6:
                    flush.zero_()  # outside the timed launch
                a.record()
                lf.backproject_batched([plan], [H], [O])
                b.record()
            torch.cuda.synchronize()
            lf.sync_status()
            return sum(a.elapsed_time(b) for a, b in ev) / reps
        t_default = time_it()
        tuned = None if no_tune else lf.tune_batched([plan], [H], [O])
        t = time_it() if tuned else t_default
        out_rows.append({"K": k, "Nx": nx, "Ny": ny, "Nz": nz, "elements": plan.elems,
                     "ms": round(t, 4), "GBps": round(world * nb / (t * 1e-3) / 1e9, 1),
                     "default_shape_GBps": round(world * nb / (t_default * 1e-3) / 1e9, 1),
                     "tuned": _tuned_desc(tuned), "paper_s": paper_s})
    del Hbuf, Obuf, flush
    torch.cuda.empty_cache()
    return {"dtype": "f32", "data": "seeded uniform values (a permutation's time does not "
                                     "depend on them)", "rows": out_rows}


def _autograd_extra(lf, timed, steps):
    """The differentiation workload: L = sum((backproject(H'(H), f) - g_ref)^2),
    forward and backward with respect to H (map, backprojection, its H'
    gradient, adjoint map), one step timed end to end on the device."""
    import torch
    import lfgen
    spec = lfgen.config_specs("autograd")[0]
    W = 64 * spec.Nx
    plan = lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, torch.float32)
    H = lfgen.generate(spec, device="cuda").requires_grad_(True)
    f = torch.from_numpy(lfgen.raw_image(64, spec.Nx, 19).astype("float32")).cuda()
    gref = torch.from_numpy(lfgen.blob_volume(W, spec.Nz, 200, 20).astype("float32")).cuda()

    def step():
        H.grad = None
        g = lf.backproject_volume(lf.backprojection_array(H, plan), f, plan)
        loss = ((g - gref) ** 2).sum()
        loss.backward()

    n = max(3, steps // 8)
    t, _, _ = timed(step, n, 3)
    return {"workload": "autograd: N=11, 21 depths, K_z 33..99, 704 x 704 image, 200-blob g_ref",
            "forward_backward_ms": round(t, 4)}


def _tuned_desc(t):
    if t is None:
        return None
    if t[4] in (1, 2):
        form = ("one tile per CTA (k_gather_tiles)" if t[4] == 1 else
                "graph of per-depth grids (k_gather_depth)")
        return {"form": form, "tile_bytes": t[0],
                "consumer": "pairs where eligible" if t[3] else "chunks / stripes"}
    return {"form": "persistent (k_gather_persistent)", "tile_bytes": t[0], "ctas_per_sm": t[1],
            "stages": t[2] or "as many as fit",
            "consumer": "pairs where eligible" if t[3] else "chunks / stripes"}


def _fp32_fma_peak_tflops():
    """Nominal fp32 CUDA-core peak: 152 SMs x 128 FMA lanes x 2 FLOP x max SM clock."""
    return 152 * 128 * 2 * 2.07e9 / 1e12


def _rl_extra(lf, timed, steps):
    """One Richardson-Lucy update (Eq. 2) on the differentiation workload (N = 11,
    21 depths, K up to 99, a 704 x 704 raw image): with H' (lfbp_rl_step) and with
    H' never built (lfbp_rl_step_fused), and H' rebuilt + update as an in-loop PSF
    update would need.  FLOP = 2 per product; products counted exactly (taps
    inside the sensor), forward and backprojection."""
    import torch
    import lfgen
    spec = lfgen.config_specs("autograd")[0]
    W = 64 * spec.Nx
    plan = lf.Plan(spec.Nx, spec.Ny, spec.Ks, spec.Kt, torch.float32)
    H = lfgen.generate(spec, device="cuda")
    Hp = lf.backproject_array(plan, H)
    f = torch.from_numpy(lfgen.raw_image(64, spec.Nx, 19).astype("float32")).cuda()
    g = torch.ones((spec.Nz, W, W), device="cuda")
    out = torch.empty_like(g)
    work = torch.empty((W, W), device="cuda")
    norm = lf.rl_normaliser(plan, H, Hp, W, W)
    norm_h = lf.rl_normaliser(plan, H, None, W, W)

    def axis(K):
        c = (K - 1) // 2
        return sum(max(0, W - abs(s - c)) for s in range(K))
    products = 2 * sum(axis(a) * axis(b) for a, b in zip(spec.Ks, spec.Kt))
    n = max(3, steps // 4)
    t_hp, _, _ = timed(lambda: lf.rl_step(plan, H, Hp, norm, f, g, out=out, work=work), n, 3)
    t_fu, _, _ = timed(lambda: lf.rl_step(plan, H, None, norm_h, f, g, out=out, work=work), n, 3)
    t_rb, _, _ = timed(lambda: (lf.backproject_array(plan, H, Hp),
                                lf.rl_step(plan, H, Hp, norm, f, g, out=out, work=work)), n, 3)
    peak = _fp32_fma_peak_tflops()
    gf = lambda ms: round(2 * products / (ms * 1e-3) / 1e9, 1)
    return {"workload": "autograd: N=11, 21 depths, K_z 33..99, 704 x 704 image, fp32",
            "products_per_step": products,
            "with_hprime_ms": round(t_hp, 4), "with_hprime_GFLOPs": gf(t_hp),
            "fused_ms": round(t_fu, 4), "fused_GFLOPs": gf(t_fu),
            "rebuild_hprime_plus_step_ms": round(t_rb, 4),
            "fp32_peak_TFLOPs": round(peak, 1), "peak_kind": "nominal 152 SM x 128 FMA x 2.07 GHz",
            "frac_fused": round(gf(t_fu) / (peak * 1e3), 4)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="weak: every rank maps its own array; strong: the ranks split the "
                         "depths of one array (lfbp_plan_partition)")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="highres",
                    choices=["tiny", "mid", "ragged", "highres", "autograd"])
    ap.add_argument("--dtype", choices=["f32", "f16"], default=None)
    ap.add_argument("--depth-stride", type=int, default=1,
                    help="keep every k-th depth only (smaller case of the same shapes)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the fp16 copy and the ragged batch beside the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the default launch shape instead of the autotuner's")
    ap.add_argument("--form", choices=["0", "1", "2"], default=None,
                    help="with --no-tune: the batched form (0 persistent CTAs, 1 one tile per "
                         "CTA, 2 per-depth grids in one graph; sets LFBP_FORM)")
    ap.add_argument("--pairs", choices=["0", "1"], default=None,
                    help="with --no-tune: the pair consumer off or on (sets LFBP_PAIRS)")
    ap.add_argument("--tile-bytes", type=int, default=None,
                    help="with --no-tune: the tile-size target (sets LFBP_TILE_BYTES)")
    ap.add_argument("--table1-rows", default=None,
                    help="with --only table1: comma-separated cut-out sizes K of the rows to time")
    ap.add_argument("--table1-depths", type=int, default=11,
                    help="with --only table1: depths per array (Table 1 has 11; fewer make a "
                         "smaller case of the same shapes)")
    ap.add_argument("--only", choices=["rl", "autograd", "table1", "window"], default=None,
                    help="time only one of the extra measurements and print that (for "
                         "profiling): the RL update (Eq. 2) or the autograd step on the "
                         "differentiation workload, the Table 1 sizes, or the paper-window "
                         "mode (odd and even cut-outs)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    # launch-shape knobs of the library, read at each call
    for flag, env in ((args.form, "LFBP_FORM"), (args.pairs, "LFBP_PAIRS"),
                      (args.tile_bytes, "LFBP_TILE_BYTES")):
        if flag is not None:
            os.environ[env] = str(flag)
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


def run_only(args):
    """One of the extra measurements alone: steps//4 timed repetitions."""
    import torch
    import paper_2003_09133_gb300 as lf
    torch.cuda.set_device(0)
    lf.load()

    def timed(fn, n, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        lf.sync_status()
        return a.elapsed_time(b) / n, None, None

    if args.only == "table1":
        rows = None if not args.table1_rows else {int(k) for k in args.table1_rows.split(",")}
        res = _table1_extra(lf, 1, args.no_tune, rows=rows, nz=args.table1_depths)
    elif args.only == "window":
        import lfgen
        args.workload = "highres"
        specs = _pick_specs(args)  # every depth_stride-th depth
        s = specs[0]
        plans = [lf.Plan(s.Nx, s.Ny, s.Ks, s.Kt, torch.float32)]
        Hs = [lfgen.generate(s, device="cuda")]
        outs = [torch.empty_like(Hs[0])]
        res = _paper_window_extra(lf, specs, Hs, outs, timed, max(3, args.steps // 4), 1,
                                  args.no_tune)
    else:
        fn = _rl_extra if args.only == "rl" else _autograd_extra
        res = fn(lf, timed, args.steps)
    print(json.dumps({"only": args.only, **res}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
