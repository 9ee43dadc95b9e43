#!/usr/bin/env python
"""Forward + backward shading throughput of the Stage-II UV-PBR renderer.

One step = one pass of the whole hot path over the workload: environment distribution
build, visibility-buffer raster, direct (+ indirect) shading, L1 loss against a target
render, and the adjoint into the maps, the environment and the vertex positions.
Metric: shaded samples per second (fwd+bwd).  One JSON line on rank 0.

The default workload is the largest single-GPU one, the precision blob (2M triangles, 8 views
of 1024^2, 64 direct + 4 x (1 + 4) indirect samples per pixel): its headline form stores the
maps and the environment in FP32, and the BF16-map / FP16-environment form is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload precision|geometry|indirect|tiny]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample (host cores)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic FP32 operation counts (per unit of work) used for the ALU roofline; an FMA counts
# 2, as in the peak, and a min, max or comparison 1
FLOPS_NODE_MODEL = 100.0  # the scope table's op model: 25 per child box slab test of a 4-wide node
FLOPS_TRI_MODEL = 30.0    # and 30 per watertight triangle test
FLOPS_NODE = 72.0       # this build's count: per child 6 FMA, a 3-way max and a max with 0, a 3-way min, one compare
FLOPS_TRI = 50.0        # one watertight test: 40 adds and multiplies (no FMA: decision arithmetic), ~10 compares
FLOPS_BRDF = 80.0       # one Lambert + GGX evaluation with its cosine and estimator weight
FLOPS_BRDF_ADJ = 240.0  # evaluation + adjoint in the backward pass
FP32_LANES_PER_SM = 128
# algorithmic bytes of the tracer: a 4-wide node record, a triangle record, a queued ray
NODE_BYTES = 128.0
TRI_BYTES = 48.0
RAY_BYTES = 32.0
# The tracer's memory traffic from one ncu capture per workload (single any-hit launch of a
# one- or two-view case of the same scene; profiles/trace_kernel_<workload>.md): DRAM bytes
# (read + write) per traced ray, L2 sector throughput and issue-slot use as fractions of peak.
TRACE_NCU = {
    "precision": {"dram_bytes_per_ray": 40.5, "l2_frac": 0.125, "issue_frac": 0.711, "l1_frac": 0.759,
                  "source": "ncu, any-hit launch of the 1-view precision case"},
}
RAY_QUEUE_MAX = 1 << 27  # rays per chunk at most (the library's default queue)
# covered pixels of the CPU-baseline sample per workload: about 10-30 s of oracle work on 16 cores
CPU_PIXELS = {"tiny": 2048, "geometry": 1536, "indirect": 384, "precision": 192}

WORKLOADS = {
    "tiny": "icosphere 1280 tris, maps 256^2 FP32, env 64x32, 4 views 256^2, 64 env samples/px, fwd+bwd",
    "geometry": "displaced blob 99,372 tris, maps 1024^2 FP32, env 256x128, 16 views 512^2, "
                "256 env samples/px, fwd+bwd to maps, env and vertex positions",
    "indirect": "blob with 3 cavities 499,392 tris, maps 2048^2 FP32, env 512x256, 8 views 800^2, "
                "128 direct + 8 secondary rays x 4 light samples/px, fwd+bwd",
    "precision": "blob with 3 cavities 1,997,568 tris, maps 4096^2, env 1024x512, 8 views 1024^2, "
                 "64 direct + 4 secondary rays x 4 light samples/px, fwd+bwd",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="precision", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-pixels", type=int, default=0,
                    help="pixels of the CPU-baseline sample (0: the workload's default)")
    ap.add_argument("--single-form", action="store_true",
                    help="precision workload: time only the --maps/--env-dtype storage form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--views", type=int, default=0, help="override the workload's view count (profiling cases)")
    ap.add_argument("--maps", default="fp32", choices=["fp32", "bf16", "fp16"], help="storage type of the UV maps")
    ap.add_argument("--env-dtype", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--relight", action="store_true", help="relight-serving benchmark (Poisson arrivals)")
    ap.add_argument("--assets", type=int, default=64)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--no-relight", action="store_true",
                    help="skip the relight-serving run the default benchmark adds to its line")
    ap.add_argument("--rate", type=float, default=200.0, help="offered requests per second")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--budget-gb", type=int, default=24)
    ap.add_argument("--half-res-indirect", action="store_true",
                    help="indirect light at half resolution, upsampled (the paper's speed variant)")
    ap.add_argument("--topology", action="store_true",
                    help="time Stage-I topology rounds on the workload's mesh (Sec. 4.1-4.3)")
    ap.add_argument("--relight-protocol", action="store_true",
                    help="relight frames/s under the paper's timing protocol (1600^2, N_d = 8, then one bounce)")
    ap.add_argument("--stage2", action="store_true",
                    help="time whole Stage-II iterations: render, objective, adjoint, Adam")
    args = ap.parse_args()
    if not args.cpu_pixels:
        args.cpu_pixels = CPU_PIXELS[args.workload]
    return args


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l.split(", ") for l in open(self.path).read().strip().splitlines() if l.count(",") >= 8]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def dist_init(timeout_s=None):
    """Joins the replicas' process group (gloo: only the timing reduction crosses ranks).  Its
    collectives give up after `timeout_s` seconds (EXM_DIST_TIMEOUT_S, default 600): a rank that
    dies or never arrives makes the others fail with an error instead of waiting forever."""
    import datetime
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        t = timeout_s if timeout_s is not None else float(os.environ.get("EXM_DIST_TIMEOUT_S", "600"))
        dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=t))
    return world, rank, local


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- CPU oracle

def oracle_sample(sc, npix, seed=0):
    """Runs the CPU oracle (decisions, FP64 radiance, autograd adjoint) on `npix` covered
    pixels of the workload.  Returns (shaded samples, seconds, threads)."""
    import numpy as np
    import torch

    import oracle
    from oracle import shade
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    # candidate pixels: random pixels, kept when the oracle's brute-force raster covers them
    pix = np.stack([rng.integers(0, sc.views, 4 * npix), rng.integers(0, sc.height, 4 * npix),
                    rng.integers(0, sc.width, 4 * npix)], 1).astype(np.int32)
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, pix)
    cov = (keys & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF)
    pix, keys = pix[cov][:npix], keys[cov][:npix]
    tab = oracle.EnvTable(sc.env)
    dec = oracle.Decisions(sc, tab, pix, keys)
    V, M, E = shade.scene_tensors(sc)
    I = shade.render_image(sc, tab, dec, V, M, E)
    g = torch.sign(I - I.mean())
    shade.backward(sc, tab, dec, V, M, E, g)
    dt = time.perf_counter() - t0
    nb = max(sc.n_bounce, 0)
    valid = int((dec.stri >= 0).sum()) if nb else 0
    samples = pix.shape[0] * (sc.n_direct + nb) + valid * sc.n_light
    return samples, dt, torch.get_num_threads(), pix.shape[0]


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2608_24109_b300 import scenes
    sc = scenes.config(args.workload)
    per_step = max(16, args.cpu_pixels // 6)
    for _ in range(args.warmup):
        oracle_sample(sc, max(4, per_step // 8), seed=99)
    times, samples = [], 0
    threads = 1
    for k in range(args.steps):
        s, dt, threads, npx = oracle_sample(sc, per_step, seed=k)
        times.append(dt)
        samples = s
    v = samples / statistics.mean(times)
    line = {"impl": "reference", "metric": "fwd+bwd shaded samples/s", "value": v, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload + ": " + WORKLOADS[args.workload],
                       "sample": f"{per_step} covered pixels per step"},
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} covered pixels of the workload per step"},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- native

def timed_steps(args, r, N, M, E, target, stream, flush, world):
    """W untimed warm-up steps, one instrumented pass (work counters), then K timed steps of the
    whole path with CUDA events on the launching stream.  Returns the per-step figures."""
    import torch

    img = torch.empty_like(target)
    grad = torch.empty_like(target)
    loss = torch.zeros(1, device=M.device)
    gm = torch.zeros(M.shape, dtype=torch.float32, device=M.device)
    gE = torch.zeros(E.shape, dtype=torch.float32, device=M.device)
    gV = torch.zeros((r.V.shape[0], 3), device=M.device)
    base_flags = r.params.flags
    r.params.flags = base_flags | N.FLAG_ZERO_GRADS

    def step(ev=None, Mx=M, Ex=E, before_loss=None):
        r.prepare_env(Ex)
        r.forward(Mx, out=img)
        if ev is not None:
            ev[0].record(stream)
        if before_loss is not None:  # the previous step's results are still being copied out
            stream.wait_event(before_loss)
        r.l1_loss(img, target, loss, grad)
        if ev is not None:
            ev[1].record(stream)
        r.backward(Mx, grad, gm, gE, gV)

    for _ in range(max(args.warmup, 0)):
        step()
    r.sync()
    covered, samples = r.stats()
    # one instrumented pass to count the algorithmic work of each shading launch
    r.params.flags = base_flags | N.FLAG_ZERO_GRADS | N.FLAG_COUNT_WORK
    r.prepare_env(E)
    r.forward(M, out=img)
    r.sync()
    work_fwd = N.exm_frame_work(r.frame)
    r.l1_loss(img, target, loss, grad)
    r.backward(M, grad, gm, gE, gV)
    r.sync()
    work_bwd = N.exm_frame_work(r.frame)
    barrier(world)
    torch.cuda.synchronize()
    N.exm_frame_kernel_ms(r.frame)  # drop timers of earlier passes
    launches0 = N.exm_launch_count(r.ctx)
    r.params.flags = base_flags | N.FLAG_ZERO_GRADS | N.FLAG_TIME_KERNELS
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    t_step, t_fwd, t_bwd = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        em = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
        e0.record(stream)
        step(em)
        e1.record(stream)
        e1.synchronize()
        t_step.append(e0.elapsed_time(e1))
        t_fwd.append(e0.elapsed_time(em[0]))
        t_bwd.append(em[1].elapsed_time(e1))
    torch.cuda.synchronize()
    ck = clocks.stop()
    kms = [x / args.steps for x in N.exm_frame_kernel_ms(r.frame)]
    r.params.flags = base_flags | N.FLAG_ZERO_GRADS
    launches = N.exm_launch_count(r.ctx) - launches0 + args.steps  # + the L1 loss kernel per step
    r.sync()
    barrier(world)
    ms = dist_max(statistics.mean(t_step), world)

    # end to end through the public API: every step's inputs (maps, environment) copied in from
    # pinned host memory and its results (loss and the gradients into maps, environment and
    # vertices) copied back.  Two schedules:
    # - serial: copy in, step, copy out, synchronise;
    # - pipelined (the headline e2e): the inputs of step k+1 are copied into a second device buffer
    #   on a copy stream while step k computes, and the results of step k are copied out on
    #   another copy stream while step k+1 runs its forward pass (step k+1's loss and backward,
    #   which overwrite the results, wait for that copy).  The time per step is the wall time of
    #   the whole pipelined run, its first copy-in and last copy-out included, over its steps.
    e2e = None
    if not args.no_e2e:
        Mh = M.cpu().pin_memory()
        Eh = E.cpu().pin_memory()
        outs = [loss, gm, gE, gV]
        hosts = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
        te = []
        for k in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            M.copy_(Mh, non_blocking=True)
            E.copy_(Eh, non_blocking=True)
            step()
            for h, t in zip(hosts, outs):
                h.copy_(t, non_blocking=True)
            torch.cuda.synchronize()
            if k >= args.warmup:
                te.append(time.perf_counter() - t0)
        serial = dist_max(statistics.mean(te), world)

        Mb, Eb = [M, torch.empty_like(M)], [E, torch.empty_like(E)]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def pipelined(n):
            in_ev = [torch.cuda.Event(), torch.cuda.Event()]
            done_ev = [torch.cuda.Event(), torch.cuda.Event()]
            out_ev = None
            with torch.cuda.stream(s_in):
                Mb[0].copy_(Mh, non_blocking=True)
                Eb[0].copy_(Eh, non_blocking=True)
                in_ev[0].record(s_in)
            for k in range(n):
                a = k & 1
                if k + 1 < n:  # prefetch the next step's inputs into the other buffer
                    with torch.cuda.stream(s_in):
                        if k >= 1:
                            s_in.wait_event(done_ev[1 - a])  # step k-1 is done with that buffer
                        Mb[1 - a].copy_(Mh, non_blocking=True)
                        Eb[1 - a].copy_(Eh, non_blocking=True)
                        in_ev[1 - a].record(s_in)
                flush.zero_()
                stream.wait_event(in_ev[a])
                step(Mx=Mb[a], Ex=Eb[a], before_loss=out_ev)
                done_ev[a].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(done_ev[a])
                    for h, t in zip(hosts, outs):
                        h.copy_(t, non_blocking=True)
                    out_ev = torch.cuda.Event()
                    out_ev.record(s_out)
            torch.cuda.synchronize()

        pipelined(max(args.warmup, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pipelined(args.steps)
        piped = dist_max((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": samples * world / piped, "unit": "samples/s",
               "h2d_bytes_per_step": Mh.numel() * Mh.element_size() + Eh.numel() * Eh.element_size(),
               "d2h_bytes_per_step": sum(h.numel() * h.element_size() for h in hosts),
               "ms_per_step": 1e3 * piped,
               "schedule": "pipelined: step k+1's inputs copied in and step k's results copied out on two copy "
                           "streams while the steps compute; first copy-in and last copy-out inside the timed run",
               "serial": {"value": samples * world / serial, "ms_per_step": 1e3 * serial,
                          "schedule": "copy in, step, copy out, synchronise, every step"}}
    r.params.flags = base_flags
    return {"ms": ms, "covered": covered, "samples": samples, "work_fwd": work_fwd, "work_bwd": work_bwd,
            "kms": kms, "clocks": ck, "launches": launches, "ms_forward": statistics.mean(t_fwd),
            "ms_backward": statistics.mean(t_bwd), "e2e": e2e, "value": samples * world / (ms * 1e-3)}


def error_table_sample(args, sc, r, M, E, mdt_name):
    """Per-output error of the GPU path against the FP64 oracle on the CPU-baseline sample:
    the oracle's decisions, radiance and adjoint on `cpu_pixels` covered pixels (the 256^2 centre
    crop of view 0 for the precision workload), the GPU's full-frame forward and its backward of
    a loss masked to those pixels.  Returns (oracle timing, error table)."""
    import numpy as np
    import torch

    import oracle
    from oracle import shade
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    n = args.cpu_pixels
    if args.workload == "precision":
        c0 = (sc.width - 256) // 2
        cand = np.stack([np.zeros(8 * n, int), rng.integers(c0, c0 + 256, 8 * n),
                         rng.integers(c0, c0 + 256, 8 * n)], 1).astype(np.int32)
    else:
        cand = np.stack([rng.integers(0, sc.views, 8 * n), rng.integers(0, sc.height, 8 * n),
                         rng.integers(0, sc.width, 8 * n)], 1).astype(np.int32)
    cand = np.unique(cand, axis=0)
    rng.shuffle(cand)
    st, keys = oracle.raster_pixels(sc.V, sc.F, sc.cams, sc.width, sc.height, cand)
    cov = (keys & np.uint64(0xFFFFFFFF)) != np.uint64(0xFFFFFFFF)
    pix, keys = cand[cov][:n], keys[cov][:n]
    import dataclasses
    sco = dataclasses.replace(sc, env=E.float().cpu().numpy())  # the environment as stored
    tab = oracle.EnvTable(sco.env)
    dec = oracle.Decisions(sco, tab, pix, keys)
    V, _, Eo = shade.scene_tensors(sco)
    Mo = M.cpu().to(torch.float64)
    I = shade.render_image(sco, tab, dec, V, Mo, Eo)
    gs = rng.normal(size=(pix.shape[0], 3))
    oV, oM, oE = shade.backward(sco, tab, dec, V, Mo, Eo, gs)
    dt = time.perf_counter() - t0
    nb = max(sc.n_bounce, 0)
    valid = int((dec.stri >= 0).sum()) if nb else 0
    samples = pix.shape[0] * (sc.n_direct + nb) + valid * sc.n_light
    threads = torch.get_num_threads()
    # the GPU on the same pixels
    img = r.forward(M, E)
    grad = torch.zeros_like(img)
    idx = tuple(torch.as_tensor(pix[:, k]).long() for k in range(3))
    grad[idx] = torch.as_tensor(gs, dtype=torch.float32, device=img.device)
    gm = torch.zeros(M.shape, dtype=torch.float32, device=M.device)
    gE = torch.zeros(E.shape, dtype=torch.float32, device=M.device)
    gV = torch.zeros((sc.V.shape[0], 3), device=M.device)
    r.backward(M, grad, gm, gE, gV)
    r.sync()

    def err(g, o):
        g = np.asarray(g, np.float64).ravel()
        o = np.asarray(o, np.float64).ravel()
        return {"max_rel": float(np.abs(g - o).max() / max(np.abs(o).max(), 1e-30)),
                "l2_rel": float(np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-30))}

    gmc = gm.cpu()
    nz = (gmc != 0).any(-1) | (oM != 0).any(-1)
    table = {"maps": mdt_name, "pixels": int(pix.shape[0]),
             "radiance": err(img[idx].cpu().numpy(), I.numpy()), "dL/dmaps": err(gmc[nz].numpy(), oM[nz].numpy()),
             "dL/dE": err(gE.cpu().numpy(), oE.numpy()), "dL/dV": err(gV.cpu().numpy(), oV.numpy())}
    return (samples, dt, threads, int(pix.shape[0])), table


def run_native(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2608_24109_b300 import build as libbuild
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.render import Renderer

    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.config(args.workload, **({"views": args.views} if args.views else {}))
    sc.half_res_indirect = args.half_res_indirect
    r = Renderer.from_scene(sc, device=local)
    dts = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # the headline form, then (precision workload) the low-precision storage form beside it
    forms = [(args.maps, args.env_dtype)]
    if args.workload == "precision" and not args.single_form:
        forms.append(("bf16", "fp16") if args.maps == "fp32" else ("fp32", "fp32"))
    res = {}
    for mname, ename in forms:
        M = torch.as_tensor(sc.maps).to(dts[mname]).to(dev).contiguous()
        E = torch.as_tensor(sc.env).to(dts[ename]).to(dev).contiguous()
        target = r.forward(torch.as_tensor(sc.maps_target).to(dts[mname]).to(dev).contiguous(), E).clone()
        res[(mname, ename)] = timed_steps(args, r, N, M, E, target, stream, flush, world)
        res[(mname, ename)]["tensors"] = (M, E)
        del target
    head = res[forms[0]]
    ms, samples, covered = head["ms"], head["samples"], head["covered"]
    value = head["value"]
    work_fwd, work_bwd, kms = head["work_fwd"], head["work_bwd"], head["kms"]

    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    trace_ms = kms[0] + kms[1]
    # the tracer's FP32 work by the op model of the scope table (25 flops per child box test of a
    # 4-wide node, 30 per watertight triangle test) and by this build's own count
    flops_model = work_fwd[0] * FLOPS_NODE_MODEL + work_fwd[1] * FLOPS_TRI_MODEL
    flops_own = work_fwd[0] * FLOPS_NODE + work_fwd[1] * FLOPS_TRI
    kinds = {
        "trace_kernel (any-hit + closest-hit)": (trace_ms, flops_model),
        "shade_kernel<forward>": (kms[2], work_fwd[2] * FLOPS_BRDF),
        "shade_kernel<backward>": (kms[3], work_bwd[2] * FLOPS_BRDF_ADJ),
    }
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_flops = kinds[dom]
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
    # the tracer's memory side: algorithmic bytes (node and triangle records fetched, the ray queue
    # read), DRAM and L2 traffic per traced ray from the ncu capture of this workload's tracer
    rays = work_fwd[3]
    algo_bytes = work_fwd[0] * NODE_BYTES + work_fwd[1] * TRI_BYTES + rays * RAY_BYTES
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    ncu = TRACE_NCU.get(args.workload)
    traffic = fractions = None
    if ncu is not None and not args.views and not args.half_res_indirect:
        fractions = {"hbm_measured": ncu["dram_bytes_per_ray"] * rays / (trace_ms * 1e-3) / (hbm * 1e9),
                     "l2_ncu": ncu["l2_frac"], "issue_slots_ncu": ncu["issue_frac"], "l1_ncu": ncu.get("l1_frac"),
                     "fp32_scope_model": flops_model / (trace_ms * 1e-3) / 1e12 / fp32_peak,
                     "fp32_own_model": flops_own / (trace_ms * 1e-3) / 1e12 / fp32_peak,
                     "algorithmic_bytes_gbs": algo_bytes / (trace_ms * 1e-3) / 1e9,
                     "source": ncu["source"]}
        if dom.startswith("trace_kernel"):
            traffic = ncu["dram_bytes_per_ray"] * rays / trace_launches(sc, args)
    config = {"workload": args.workload + ": " + WORKLOADS[args.workload],
              "map_storage": forms[0][0], "env_storage": forms[0][1], "covered_pixels": covered,
              "shaded_samples_per_step": samples,
              "indirect_resolution": "half, upsampled" if args.half_res_indirect else "full",
              "l2": "flushed between steps (256 MiB write outside the timed region)",
              "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
              "ms_forward": head["ms_forward"], "ms_backward": head["ms_backward"],
              "kernel_ms_per_step": {"trace_any": kms[0], "trace_closest": kms[1], "shade_forward": kms[2],
                                     "shade_backward": kms[3]},
              "work_per_step": {"nodes": work_fwd[0], "tri_tests": work_fwd[1], "rays": work_fwd[3],
                                "brdf_fwd": work_fwd[2], "brdf_bwd": work_bwd[2]}}
    for key, rr in res.items():
        if key == forms[0]:
            continue
        config["other_storage_form"] = {
            "map_storage": key[0], "env_storage": key[1], "value": rr["value"], "ms_per_step": rr["ms"],
            "ratio_to_headline": rr["value"] / value,
            "kernel_ms_per_step": {"trace_any": rr["kms"][0], "trace_closest": rr["kms"][1],
                                   "shade_forward": rr["kms"][2], "shade_backward": rr["kms"][3]},
            "e2e": rr["e2e"], "clocks": rr["clocks"]}
    line = {
        "metric": "fwd+bwd shaded samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic,
                     "traffic_unit": "bytes per any-hit launch (ncu DRAM read + write per traced ray x rays per launch)",
                     "peak_source": f"FP32 FMA: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz "
                                    f"(clock from {src} peaks)",
                     "op_model": f"{FLOPS_NODE_MODEL:.0f} flops per 4-wide node visit, {FLOPS_TRI_MODEL:.0f} per "
                                 "triangle test (scope table); own count "
                                 f"{FLOPS_NODE:.0f} / {FLOPS_TRI:.0f}",
                     "fractions": fractions},
        "clocks": head["clocks"],
        "gpu_launches": head["launches"],
    }
    if head["e2e"]:
        line["e2e"] = head["e2e"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the CPU baseline is an N = 1 figure
        tables = []
        for key in forms:
            M, E = res[key]["tensors"]
            (s, dt, threads, npx), table = error_table_sample(args, sc, r, M, E, key[0])
            tables.append(table)
            if key == forms[0]:
                line["cpu_baseline"] = {"value": s / dt, "unit": "samples/s", "cores": threads, "kind": "oracle",
                                        "sample": f"{npx} covered pixels of the workload"
                                                  f"{' (256^2 centre crop of view 0)' if args.workload == 'precision' else ''}: "
                                                  f"decisions, FP64 radiance and adjoint, {dt:.1f} s"}
        line["error_vs_oracle"] = tables
    r.close()
    if rank == 0 and world == 1 and not args.no_relight:
        # relight serving beside the training-step throughput: the 64-asset mix at 200 req/s
        rl = run_relight(args, world, rank, local, emit=False)
        line["relight"] = {k: rl[k] for k in ("p50_ms", "p99_ms", "mean_ms", "frames_per_s", "offered_req_per_s",
                                              "requests")}
        line["relight"]["config"] = rl["config"]
        line["relight"]["clocks"] = rl["clocks"]
    if rank == 0:
        print(json.dumps(line), flush=True)


def trace_launches(sc, args):
    """Any-hit tracer launches per forward pass: one per ray-queue chunk."""
    per_pixel = ((sc.n_direct + 31) // 32) * 32
    if sc.n_bounce > 0:
        per_pixel += ((sc.n_bounce * sc.n_light + 31) // 32) * 32
    pixels = sc.views * sc.width * sc.height
    chunk = max(32, min((pixels + 31) & ~31, (RAY_QUEUE_MAX // per_pixel) & ~31))
    return -(-pixels // chunk)


def run_stage2(args, world, rank, local):
    """Stage-II iterations (Sec. 5.4): forward render, image term (log-L1 + D-SSIM), adjoint,
    material TV, environment TV and chroma, Adam on the maps and the environment."""
    import numpy as np
    import torch

    from paper_2608_24109_b300 import build as libbuild
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.objective import ENV_HI, ENV_LO, MAP_HI, MAP_LO, Stage2Optimizer
    from paper_2608_24109_b300.render import Renderer

    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.config(args.workload, **({"views": args.views} if args.views else {}))
    r = Renderer.from_scene(sc, device=local)
    M = torch.as_tensor(sc.maps).to(dev)
    E = torch.as_tensor(sc.env).to(dev)
    target = r.forward(torch.as_tensor(sc.maps_target).to(dev), E).clone()
    opt = Stage2Optimizer(r, M, E, total_steps=args.warmup + args.steps)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def iteration(ev):
        # Stage2Optimizer.step with events between its phases
        r.forward(opt.maps, opt.env, out=opt.image)
        ev[0].record(stream)
        N.exm_image_loss(r.ctx, opt.image, target, opt.lambda_ssim, opt.loss[0:3], opt.grad_rgb)
        ev[1].record(stream)
        opt.grad_maps.zero_()
        opt.grad_env.zero_()
        r.backward(opt.maps, opt.grad_rgb, opt.grad_maps, opt.grad_env, None)
        ev[2].record(stream)
        N.exm_material_tv(r.ctx, opt.maps, r.frame, r.params.flags, opt.lambda_mat, opt.loss[3:4], opt.grad_maps)
        opt.last_lambda_chroma = opt.lambda_chroma()
        N.exm_env_regularizers(r.ctx, opt.env, opt.lambda_env, opt.last_lambda_chroma, opt.loss[4:6], opt.grad_env)
        ev[3].record(stream)
        opt.t += 1
        N.exm_adam_step(r.ctx, opt.maps, opt.grad_maps, opt.m_maps, opt.v_maps, opt.lr_maps, opt.t, MAP_LO, MAP_HI)
        N.exm_adam_step(r.ctx, opt.env, opt.grad_env, opt.m_env, opt.v_env, opt.lr_env, opt.t, ENV_LO, ENV_HI)

    def events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    for _ in range(max(args.warmup, 0)):
        ev = events()
        iteration(ev[1:5])
    r.sync()
    first_loss = opt.total_loss()
    covered, samples = r.stats()
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = N.exm_launch_count(r.ctx)
    clocks.start()
    parts = {"render_forward": [], "image_loss": [], "render_backward": [], "regularizers": [], "adam": [],
             "iteration": []}
    for _ in range(args.steps):
        flush.zero_()
        ev = events()
        ev[0].record(stream)
        iteration(ev[1:5])
        ev[5].record(stream)
        ev[5].synchronize()
        for k, name in enumerate(["render_forward", "image_loss", "render_backward", "regularizers", "adam"]):
            parts[name].append(ev[k].elapsed_time(ev[k + 1]))
        parts["iteration"].append(ev[0].elapsed_time(ev[5]))
    torch.cuda.synchronize()
    ck = clocks.stop()
    launches = N.exm_launch_count(r.ctx) - launches0
    r.sync()
    barrier(world)
    ms = dist_max(statistics.mean(parts["iteration"]), world)
    ms_loss = statistics.mean(parts["image_loss"])
    # image term: pred and target read by three kernels, the gradient written and updated, and the
    # three SSIM coefficient planes written and read (4-byte values)
    n_val = r.views * r.width * r.height * 3
    loss_bytes = n_val * 4 * (2 * 3 + 1 + 2 + 3 * 2)
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    line = {
        "metric": "Stage-II iterations/s", "value": world * 1e3 / ms, "unit": "iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload + ": " + WORKLOADS[args.workload] + "; Stage-II objective "
                               "(log-L1 + 0.2 D-SSIM, material TV, env TV, chroma) and Adam on maps and env",
                   "covered_pixels": covered, "shaded_samples_per_iteration": samples,
                   "l2": "flushed between iterations (256 MiB write outside the timed region)",
                   "ms_parts": {k: statistics.mean(v) for k, v in parts.items() if k != "iteration"},
                   "objective_first": first_loss, "objective_last": opt.total_loss()},
        "roofline": {"bound": "hbm", "kernel": "exm_image_loss (log-L1 + SSIM forward + SSIM adjoint)",
                     "achieved": loss_bytes / (ms_loss * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": loss_bytes / (ms_loss * 1e-3) / 1e9 / hbm, "traffic": None,
                     "peak_source": f"{src} HBM copy bandwidth"},
        "clocks": ck,
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    r.close()


def run_topology(args, world, rank, local):
    """Stage-I topology rounds (EMA, scores, greedy splits and collapses, UV maintenance,
    compaction) on the workload's mesh; render counts from a raster of its views."""
    import numpy as np
    import torch

    from paper_2608_24109_b300 import build as libbuild
    from paper_2608_24109_b300 import native as N
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.render import Renderer
    from paper_2608_24109_b300.topology import TopologyRound

    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.config(args.workload, **({"views": args.views} if args.views else {}))
    r = Renderer.from_scene(sc, device=local)
    r.forward(torch.as_tensor(sc.maps).to(dev), torch.as_tensor(sc.env).to(dev))
    nf = sc.F.shape[0]
    counts = torch.zeros(nf, dtype=torch.int32, device=dev)
    N.exm_face_render_counts(r.frame, nf, counts)
    rng = np.random.default_rng(0)
    V = torch.as_tensor(sc.V, device=dev)
    F = torch.as_tensor(sc.F, device=dev)
    UV = torch.as_tensor(sc.UV, device=dev)
    Fuv = torch.as_tensor(sc.Fuv, device=dev)
    G = torch.as_tensor(rng.uniform(0, 1, sc.V.shape[0]).astype(np.float32), device=dev)
    grad = torch.as_tensor(rng.normal(size=sc.V.shape).astype(np.float32), device=dev)
    tr = TopologyRound(r.ctx)
    for _ in range(max(args.warmup, 1)):
        out, stats = tr(V, F, UV, Fuv, G, grad, counts)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    launches0 = N.exm_launch_count(r.ctx)
    clocks.start()
    times = []
    stream = torch.cuda.current_stream()
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out, stats = tr(V, F, UV, Fuv, G, grad, counts)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ck = clocks.stop()
    launches = (N.exm_launch_count(r.ctx) - launches0) // max(args.steps, 1)
    ms = dist_max(statistics.mean(times), world)
    line = {"metric": "Stage-I topology round, input faces/s", "value": world * nf / (ms * 1e-3), "unit": "faces/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload} mesh: {nf} faces, {sc.V.shape[0]} vertices, {sc.UV.shape[0]} UVs; "
                                   "one round: EMA, curvature and split scores, splits of 5% of the faces, collapses "
                                   "of small degenerate or never-rendered faces, UV maintenance, compaction",
                       "render_counts": f"from a raster of the workload's {sc.views} views",
                       "faces_out": int(out[1].shape[0]), **stats, "kernel_launches_per_round": int(launches),
                       "note": "synchronous: the host reads sizes and selection state back between rounds of the "
                               "greedy selection"},
            "clocks": ck}
    if rank == 0:
        print(json.dumps(line), flush=True)
    tr.close()
    r.close()


def run_relight(args, world, rank, local, emit=True):
    """Relight serving: Poisson arrivals of relight renders over resident assets."""
    import math

    import numpy as np
    import torch

    from paper_2608_24109_b300 import build as libbuild
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.serve import RelightServer

    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(5)
    srv = RelightServer(hbm_budget_bytes=args.budget_gb << 30, max_slots=args.slots, device=local)
    ids, tris = [], []
    for a in range(args.assets):
        t = math.exp(rng.uniform(math.log(1e4), math.log(2e6)))
        n = max(8, int(round(math.sqrt(t / 12.0))))
        res = int(rng.choice([512, 1024, 2048, 4096]))
        ra = np.random.default_rng(1000 + a)
        V, F, UV, Fuv = scenes.cube_sphere(n, res, ra, dents=int(ra.integers(0, 4)))
        maps = torch.as_tensor(scenes.material_maps(ra, res)).to(torch.bfloat16)
        ids.append(srv.add_asset(V, F, UV, Fuv, maps))
        tris.append(F.shape[0])
    envs = [torch.as_tensor(scenes.env_map(np.random.default_rng(w + v), w, h, 1.5), device=dev)
            for (w, h) in [(256, 128), (512, 256), (1024, 512)] for v in range(2)]

    def make(k):
        r2 = np.random.default_rng(10_000 + k)
        res = int(r2.choice([256, 512, 1024]))
        d = r2.normal(size=3)
        d = 3.0 * d / np.linalg.norm(d)
        cams = np.stack([scenes.look_at_camera(d, res, res)])
        return srv.request(ids[int(r2.integers(0, len(ids)))], envs[int(r2.integers(0, len(envs)))], cams, res, res,
                           n_direct=64, n_bounce=4, n_light=4, seed=k)

    total = args.warmup * 8 + args.requests
    gaps = np.random.default_rng(6).exponential(1.0 / args.rate, total)
    arrivals = np.cumsum(gaps)
    reqs = [make(k) for k in range(total)]
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    inflight, lat, done_at = {}, {}, {}
    nxt = 0
    while len(lat) < total:
        now = time.perf_counter() - t0
        while nxt < total and arrivals[nxt] <= now:
            inflight[srv.submit(reqs[nxt])] = nxt
            nxt += 1
        for tk in list(inflight):
            d, _, _ = srv.poll(tk)
            if d:
                k = inflight.pop(tk)
                tnow = time.perf_counter() - t0
                lat[k] = 1e3 * (tnow - arrivals[k])
                done_at[k] = tnow
    torch.cuda.synchronize()
    ck = clocks.stop()
    batches, batched = srv.batches()
    meas = list(range(args.warmup * 8, total))
    L = np.array([lat[k] for k in meas])
    span = max(done_at[k] for k in meas) - arrivals[meas[0]]
    line = {"metric": "relight latency p99 (p50 beside) at offered rate", "value": float(np.percentile(L, 99)),
            "unit": "ms", "higher_is_better": False, "p50_ms": float(np.percentile(L, 50)),
            "p99_ms": float(np.percentile(L, 99)), "mean_ms": float(L.mean()), "frames_per_s": len(meas) / span,
            "offered_req_per_s": args.rate, "requests": len(meas), "warmup_requests": args.warmup * 8,
            "n_gpus": 1, "dtype": "bf16 maps, f32 shading", "data": "synthetic",
            "config": {"workload": f"relight serving: {args.assets} resident assets, 10K-2M tris (log-uniform, "
                                   f"{min(tris)}-{max(tris)}), maps 512^2-4096^2 BF16, env 256x128-1024x512, "
                                   f"outputs 256^2-1024^2, 64 direct + 4 secondary x 4 light samples/px, Poisson "
                                   f"arrivals", "slots": args.slots, "hbm_budget_gb": args.budget_gb,
                       "batching": f"{batched} requests in {batches} batches (persistent tracer launches shared "
                                   "by the requests of a batch)"},
            "clocks": ck}
    srv.close()
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_relight_protocol(args, world, rank, local):
    """Relight frames under the paper's relighting timing protocol (Sec. 6.6): the first frame
    is a warm-up; each timed frame includes the environment's transfer from pinned host memory,
    its sampling distribution, light transport and shading; asset loading is not timed.  The
    asset is the geometry blob (99,372 tris, ~50K vertices) with BF16 maps 1024^2, one view at
    1600 x 1600, a new 512 x 256 environment per frame; N_d = 8 direct samples, then the same
    with one bounce (N_b = 16 secondary rays at half resolution, N_s = 4)."""
    import numpy as np
    import torch

    from paper_2608_24109_b300 import build as libbuild
    from paper_2608_24109_b300 import scenes
    from paper_2608_24109_b300.render import Renderer

    libbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scenes.config("geometry")
    W = H = 1600
    cams = np.stack([scenes.look_at_camera((0.0, 0.4, 3.0), W, H)])
    maps = torch.as_tensor(sc.maps).to(torch.bfloat16).to(dev).contiguous()
    envs = [torch.as_tensor(scenes.env_map(np.random.default_rng(40 + k), 512, 256, 1.5)).pin_memory() for k in range(4)]
    frames = max(args.steps, 10)
    results = {}
    for name, kw in [("direct", dict(n_direct=8)),
                     ("one_bounce", dict(n_direct=8, n_bounce=16, n_light=4, half_res_indirect=True))]:
        r = Renderer(sc.V, sc.F, sc.UV, sc.Fuv, 512, 256, cams, W, H, seed=7, device=local, **kw)
        Ed = torch.empty((256, 512, 3), dtype=torch.float32, device=dev)
        out = torch.empty(r.image_shape(), dtype=torch.float32, device=dev)
        times = []
        for f in range(frames + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Ed.copy_(envs[f % len(envs)], non_blocking=True)
            r.forward(maps, Ed, out=out)
            r.sync()
            if f > 0:
                times.append(time.perf_counter() - t0)
        covered, _ = r.stats()
        results[name] = {"frames_per_s": 1.0 / statistics.mean(times), "ms_per_frame": 1e3 * statistics.mean(times),
                         "covered_pixels": int(covered)}
        r.close()
    line = {"metric": "relight frames/s (paper's protocol)", "value": results["direct"]["frames_per_s"],
            "unit": "frames/s", "higher_is_better": True, "n_gpus": 1, "frames": frames, "vs_baseline": None,
            "dtype": "bf16 maps, f32 shading", "data": "synthetic",
            "config": {"workload": "geometry blob 99,372 tris, BF16 maps 1024^2, env 512x256 new per frame, "
                                   "1 view 1600x1600, N_d = 8; one bounce: N_b = 16 at half resolution, N_s = 4",
                       "timed": "env upload from pinned host memory + env distribution + render, per frame"},
            "direct": results["direct"], "one_bounce": results["one_bounce"],
            "context": "paper, RTX A6000, Stanford-ORB 1600^2: 40.47 frames/s direct-only, 15.09 with one bounce "
                       "(other hardware and assets; not a ratio)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.relight:
        if rank == 0:
            run_relight(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    elif args.relight_protocol:
        if rank == 0:
            run_relight_protocol(args, world, rank, local)
    elif args.stage2:
        run_stage2(args, world, rank, local)
    elif args.topology:
        run_topology(args, world, rank, local)
    else:
        run_native(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
