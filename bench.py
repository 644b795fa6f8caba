#!/usr/bin/env python
"""Throughput of the forward + adjoint path trace (path segments per second).

One step = forward render of every view of the workload, the L2 image-loss
gradient against a resident target, and the adjoint (path replay for the
interior term plus silhouette edge sampling). A path segment is one BVH ray
query (extension, shadow or edge-side). Default workload: 64 views of uneven
resolution ({64,128,256,512}^2) and spp ({1,4,16}) of a 200,000-face displaced
sphere under a 512x256 environment, 3 bounces, batched persistent launches
replayed from CUDA graphs; the plain per-view launch path is timed beside it.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded pixel sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fwd+adjoint path segments/s (M/s), batched vs per-view, at grad rel err ≤1e-3"
UNIT = "Mseg/s"
DESCRIPTIONS = {
    "batched": ("batched uneven views: displaced UV sphere 200000 faces, per-face Torrance-Sparrow (GGX), env 512x256 "
                "lognormal(0,1.5), 64 Fibonacci-sphere views with W,H in {64,128,256,512} and spp in {1,4,16}, "
                "3 bounces; forward + adjoint (interior replay + silhouette edge term)"),
    "tiny": ("tiny: icosphere 320 faces, 1 point light, one 64x64 view, 4 spp, 2 bounces; forward + adjoint "
             "(interior + silhouette edges)"),
    "edges": ("edges: displaced icosphere 5120 faces, 3 point lights, 16 ring views 128x128, 16 spp, 3 bounces; "
              "forward + adjoint (interior + silhouette edges)"),
    "env": ("env: torus knot 50000 faces, env 256x128 lognormal(0,1.5), 32 views 256x256, 4 spp, 4 bounces; "
            "forward + interior adjoint with path replay"),
    "scale": ("scale: fractal-displaced UV sphere 1000000 faces, env 1024x512 + 2 point lights, 100 views 512x512, "
              "16 spp, 5 bounces; one step = one Adam iteration over an 8-view minibatch (BVH refit, forward, "
              "MSE, adjoint with interior + silhouette edges, Adam update at zero learning rate)"),
    "color_bleed": ("color_bleed: three intersecting planes (red, blue, white floor) of 384 faces, 1 point light, "
                    "4 views 64x64, 16 spp, 3 bounces; forward + adjoint (interior + silhouette edges)"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--per-view-steps", type=int, default=0, help="0 = max(2, steps // 3)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--views", type=int, default=0, help="profiling: keep only the first N views")
    ap.add_argument("--chunk", type=int, default=0, help="paths in flight per wavefront chunk (0 = library default)")
    ap.add_argument("--bvh", default="ploc", choices=["ploc", "lbvh"], help="tree builder")
    ap.add_argument("--profile", action="store_true",
                    help="profiling driver: warm-up steps then one batched fwd+adjoint step, no JSON")
    return ap.parse_args()


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------------------- CPU oracle leg
def oracle_sample_rate(sc, seconds, seed=2024, max_views=4, threads=0):
    """Segments/s of the FP64 oracle (forward + interior gradient + edge term) on a pixel sample."""
    import oracle as O
    rng = np.random.default_rng(seed)
    if len(sc.views) > max_views:
        sc = sc.subset_views(sorted(rng.choice(len(sc.views), size=max_views, replace=False)))
    osc = O.OracleScene(sc)
    npix = 4
    cores = threads or os.cpu_count() or 1
    t_total, seg_total, pix_total = 0.0, 0, 0
    while True:
        vi = rng.integers(len(sc.views), size=npix)
        pix = np.array([(v, rng.integers(sc.views[v].width), rng.integers(sc.views[v].height)) for v in vi], np.int32)
        rows = O.pixel_index(sc, pix)
        w = np.zeros((sc.n_pixels, 3))
        w[rows] = rng.normal(size=(len(pix), 3))
        prm = O.params(sc.max_bounces, seed, edge_mode=0, n_threads=cores)
        t0 = time.perf_counter()
        _, s1 = O.render_pixels(osc, prm, pix)
        _, _, s2 = O.grad_pixels(osc, prm, pix, w[rows])
        _, s3 = O.edge_grad(osc, prm, w)
        dt = time.perf_counter() - t0
        t_total += dt
        seg_total += s1 + s2 + s3
        pix_total += len(pix)
        if t_total >= seconds:
            break
        npix = int(min(4096, max(npix * 2, npix * (seconds - t_total) / max(dt, 1e-3) * 0.5)))
    return seg_total / t_total / 1e6, cores, pix_total, t_total


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    from paper_2012_03939_gb300 import scenes as S
    import oracle as O
    O.build()
    sc = S.make(args.workload)
    per_step = max(2.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_rate(sc, per_step / 4)
    rates, cores, pix = [], 0, 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        r, cores, p, _ = oracle_sample_rate(sc, per_step, seed=100 + k)
        rates.append(r)
        pix += p
    wall = time.perf_counter() - t0
    v = statistics.mean(rates)
    sample = "%d sampled pixels over %d steps: forward + interior gradient + edge term, brute-force FP64" % (
        pix, args.steps)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * wall / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": DESCRIPTIONS[args.workload], "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def secondary_on_torus_knot(st, S, chunk, persist, n_views=8, steps=4):
    """The step with and without the secondary-visibility edge term on the concave torus knot (8 of its
    256x256 views, 4 spp, 4 bounces, silhouette primary term on), where path vertices see silhouettes."""
    import torch
    sc = S.env().subset_views(range(n_views))
    B, seed = sc.max_bounces, 515
    scn = st.Scene.from_scene(sc)
    img = torch.zeros((sc.n_pixels, 3), dtype=torch.float32, device="cuda")
    g = torch.full((sc.n_pixels, 3), 1e-3, dtype=torch.float32, device="cuda")
    fo = st.make_opts(mode="batched", use_graph=1, chunk_paths=chunk, persist_blocks=persist)
    out = {"workload": "torus knot 50000 faces, env 256x128, %d views 256x256, 4 spp, 4 bounces" % n_views}
    for name, term in (("primary", st.EDGE_TERM_PRIMARY), ("primary+secondary",
                                                            st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SECONDARY)):
        bo = st.make_opts(mode="batched", use_graph=1, edge_term=term, edge_mode=0, chunk_paths=chunk,
                          persist_blocks=persist, sec_pick="tree")

        def one():
            scn.render(sc.views, B, seed, fo, out=img)
            scn.backward(sc.views, B, seed, g, bo)

        one()
        s0 = scn.stats()
        scn.render(sc.views, B, seed, fo, out=img)
        s1 = scn.stats()
        segs = s0["extension_rays"] + s0["shadow_rays"] + s1["extension_rays"] + s1["shadow_rays"]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            one()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": round(ms, 3), "segments_per_step": segs,
                     "value": round(segs / (ms / 1000.0) / 1e6, 3), "secondary_samples_per_step": s0["secondary_samples"]}
    scn.close()
    assert out["primary+secondary"]["secondary_samples_per_step"] > 0, "the secondary term drew no sample"
    out["cost"] = round(out["primary+secondary"]["ms_per_step"] / out["primary"]["ms_per_step"] - 1.0, 4)
    return out


def oracle_parity(st, scene, sc, target, B, seed, fopts, bopts, edge_on, n_img=1024, n_grad=256):
    """Checks the timed launch configuration against the FP64 oracle on seeded pixel samples: image values
    and path signatures; the interior gradient of the step's L2 loss restricted to a pixel sample (relative
    L2 over vertices and texel parameters: the metric's gradient error); the silhouette edge term on the same
    sample against the oracle's estimator with identical samples."""
    import torch
    import oracle as O
    t0 = time.perf_counter()
    rng = np.random.default_rng(31)

    def sample(n):
        vi = rng.integers(len(sc.views), size=n)
        pix = np.array([(v, rng.integers(sc.views[v].width), rng.integers(sc.views[v].height)) for v in vi], np.int32)
        return np.unique(pix, axis=0)

    N = sc.n_pixels
    sig = torch.zeros(N, dtype=torch.int64, device="cuda")
    img = scene.render(sc.views, B, seed, fopts, signatures=sig)
    sig = sig.cpu().numpy().view(np.uint64)
    osc = O.OracleScene(sc)
    prm = O.params(B, seed, edge_mode=0)
    pix = sample(n_img)
    rows = O.pixel_index(sc, pix)
    ref, _ = O.render_pixels(osc, prm, pix)
    rsig = O.render_signatures(osc, prm, pix)
    g = img.cpu().numpy()[rows].astype(np.float64)
    err = np.abs(g - ref)
    ok = err <= 1e-4 * np.abs(ref) + 1e-7
    same = sig[rows] == rsig
    out = {"pixels": int(len(pix)), "channels_within_1e-4": round(float(ok.mean()), 5),
           "mean_rel_err": float(err.mean() / np.abs(ref).mean()), "signatures_equal": round(float(same.mean()), 5),
           "out_of_tolerance_with_equal_signatures": int((~np.all(ok, 1) & same).sum())}
    # the step's loss gradient dL/dI = 2 (I - target) / (3N), kept on a pixel sample
    gp = sample(n_grad)
    grows = O.pixel_index(sc, gp)
    dLdI = ((img - target) * (2.0 / (3 * N))).cpu().numpy()
    w = np.zeros_like(dLdI)
    w[grows] = dLdI[grows]
    wt = torch.from_numpy(w).cuda()
    o_int = st.RenderOpts.from_buffer_copy(bopts)
    o_int.edge_term = 0
    dVi, dFi = scene.backward(sc.views, B, seed, wt, o_int)
    rv, rf, _ = O.grad_pixels(osc, prm, gp, w[grows].astype(np.float64))
    got = np.concatenate([dVi.cpu().numpy().ravel(), dFi.cpu().numpy().ravel()]).astype(np.float64)
    exp = np.concatenate([rv.ravel(), rf.ravel()])
    out["grad_pixels"] = int(len(gp))
    out["grad_rel_err"] = float(np.linalg.norm(got - exp) / np.linalg.norm(exp))
    # the same over the pixels whose paths took the oracle's decisions (equal path signatures): what is left
    # when the few paths where FP32 and FP64 decided differently are set aside
    gsame = sig[grows] == O.render_signatures(osc, prm, gp)
    out["grad_pixels_diverged"] = int((~gsame).sum())
    if (~gsame).any():
        w2 = np.zeros_like(dLdI)
        w2[grows[gsame]] = dLdI[grows[gsame]]
        dV2, dF2 = scene.backward(sc.views, B, seed, torch.from_numpy(w2).cuda(), o_int)
        rv2, rf2, _ = O.grad_pixels(osc, prm, gp[gsame], w2[grows[gsame]].astype(np.float64))
        g2 = np.concatenate([dV2.cpu().numpy().ravel(), dF2.cpu().numpy().ravel()]).astype(np.float64)
        e2 = np.concatenate([rv2.ravel(), rf2.ravel()])
        out["grad_rel_err_equal_signatures"] = float(np.linalg.norm(g2 - e2) / np.linalg.norm(e2))
    else:
        out["grad_rel_err_equal_signatures"] = out["grad_rel_err"]
    if edge_on:
        dVe, _ = scene.backward(sc.views, B, seed, wt, bopts)
        ev, _ = O.edge_grad(osc, prm, w.astype(np.float64))
        ge = (dVe - dVi).cpu().numpy().astype(np.float64)
        out["edge_rel_err"] = float(np.linalg.norm(ge - ev) / max(np.linalg.norm(ev), 1e-300))
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- ours
def source_hash():
    h = hashlib.sha256()
    for f in ("st_trace.cuh", "st_kernels.cuh", "st_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2012_03939_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per closest-hit and per any-hit query from the committed ncu summary, if taken on the current
    traversal sources (else None, None)."""
    p = os.path.join(ROOT, "profiles", "traversal_dram_traffic_batched_8views.txt")
    if not os.path.exists(p):
        return None, None
    kv = {}
    for ln in open(p):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != source_hash():
        return None, None
    return float(kv["extend_dram_bytes_per_query"]), float(kv["shadow_dram_bytes_per_query"])


def l2_peak_gbs(st):
    """Best of a few sizes of the library's L2-resident read probe (GB/s)."""
    return max(st.measure_l2_read(mb << 20, 64) for mb in (16, 32, 48))


def run_ours(args):
    import torch
    from paper_2012_03939_gb300 import build as Bld
    from paper_2012_03939_gb300 import scenes as S
    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        Bld.build()
    if world > 1:
        dist.barrier()
    from paper_2012_03939_gb300 import st
    from paper_2012_03939_gb300.dist import max_over_ranks

    sc = S.make(args.workload)
    if args.views:
        sc = sc.subset_views(range(args.views))
    B = sc.max_bounces
    t_build = time.perf_counter()
    scene = st.Scene.from_scene(sc, bvh_builder=args.bvh)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    views = sc.views
    N = sc.n_pixels
    seed = 20240 + rank
    # resident target: the same views rendered from a perturbed copy of the mesh
    noisy = sc.vertices + np.random.default_rng(7).normal(0, 0.01, sc.vertices.shape).astype(np.float32)
    tgt_scene = st.Scene.from_scene(sc, vertices=noisy)
    target = tgt_scene.render(views, B, 99)
    torch.cuda.synchronize()
    tgt_scene.close()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    img = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    dV = torch.zeros((scene.nv, 3), dtype=torch.float32, device="cuda")
    dF = torch.zeros(tuple(scene.face_params.shape), dtype=torch.float32, device="cuda")
    inv_n = 1.0 / (3 * N)

    adam = args.workload == "scale"
    if adam:
        # one step = one Adam iteration over an 8-view minibatch (refit, render, MSE, adjoint, update)
        import dataclasses
        from paper_2012_03939_gb300 import optimize as Opt
        rec = Opt.Reconstruction(scene, views, target, torch.from_numpy(sc.vertices).cuda(),
                                 torch.from_numpy(sc.face_params).cuda(),
                                 # zero learning rates: every step still refits, renders, differentiates
                                 # and runs the Adam arithmetic, but the mesh stays the one whose ray
                                 # queries were counted, so the segment count is exact for every step
                                 Opt.AdamConfig(max_bounces=B, minibatch=8, edge_term=1, seed=seed,
                                                lr_vertices=0.0, lr_params=0.0))
        step_views, off = [], 0
        for v in views[:8]:
            step_views.append(dataclasses.replace(v, pixel_offset=off))
            off += v.width * v.height
        Ns = off
        img = torch.zeros((Ns, 3), dtype=torch.float32, device="cuda")
        step_target = target[:Ns]
    else:
        step_views, Ns, step_target = views, N, target
    inv_s = 1.0 / (3 * Ns)

    def new_vertices(scn):
        # an optimisation iteration renders updated vertices: the refit (on the same vertices here, so that the
        # ray counts stay exact) makes every step redo what depends on them, the BVH boxes and the
        # primary-visibility lists, which calls on unchanged vertices and views would otherwise reuse
        scn.refit(scn.vertices)

    def step(fopts, bopts):
        if adam:
            rec.fopts, rec.bopts = fopts, bopts
            rec.step()
            return
        new_vertices(scene)
        scene.render(views, B, seed, fopts, out=img)
        g = (img - target) * (2 * inv_n)
        dV.zero_()
        dF.zero_()
        scene.backward(views, B, seed, g, bopts, d_vertices=dV, d_face_params=dF)

    def counts(fopts, bopts):
        new_vertices(scene)
        scene.render(step_views, B, seed, fopts, out=img)
        a = scene.stats()
        g = (img - step_target) * (2 * inv_s)
        scene.backward(step_views, B, seed, g, bopts, d_vertices=dV, d_face_params=dF)
        b = scene.stats()
        return a, b

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.fill_(1.0)            # evict L2 (256 MiB > 129 MB) between timed steps
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        return max_over_ranks(ms, device="cuda")

    edge_on = 0 if args.workload == "env" else 1     # the environment workload is forward + interior adjoint
    tuned = None
    chunk, persist = args.chunk, 0
    if not args.chunk and not args.profile:
        from paper_2012_03939_gb300 import autotune
        tuned = autotune.tune(scene, step_views, B, seed, edge_term=edge_on, edge_mode=0,
                              cache_path=os.path.join(tempfile.gettempdir(), "st_autotune_cache.rank%d.json" % rank))
        chunk, persist = tuned["chunk_paths"], tuned["persist_blocks"]
    fb = st.make_opts(mode="batched", use_graph=1, chunk_paths=chunk, persist_blocks=persist)
    bb = st.make_opts(mode="batched", use_graph=1, edge_term=edge_on, edge_mode=0, chunk_paths=chunk,
                      persist_blocks=persist)
    if args.profile:
        for _ in range(args.warmup):
            step(fb, bb)
        torch.cuda.synchronize()
        new_vertices(scene)
        scene.render(views, B, seed, fb, out=img)
        torch.cuda.synchronize()
        sf = scene.stats()
        g = (img - target) * (2 * inv_n)
        scene.backward(views, B, seed, g, bb, d_vertices=dV, d_face_params=dF)
        torch.cuda.synchronize()
        s = scene.stats()
        print("profile step done: %d + %d kernel launches, %d + %d closest-hit and %d + %d any-hit queries "
              "(forward + adjoint), device_error %d" % (sf["kernel_launches"], s["kernel_launches"],
                                                         sf["extension_rays"], s["extension_rays"],
                                                         sf["shadow_rays"], s["shadow_rays"], s["device_error"]))
        scene.close()
        return
    fp = st.make_opts(mode="per_view", use_graph=0)
    bp = st.make_opts(mode="per_view", use_graph=0, edge_term=edge_on, edge_mode=0)

    sf, sb = counts(fb, bb)
    seg_fwd = sf["extension_rays"] + sf["shadow_rays"]
    seg_step = seg_fwd + sb["extension_rays"] + sb["shadow_rays"]
    # + the refit of every step (bottom-up boxes, 4-wide boxes, three mesh-statistics kernels) and, in an Adam
    # iteration, the upload of the face parameters
    launches_step = sf["kernel_launches"] + sb["kernel_launches"] + (6 if adam else 5)
    assert sf["device_error"] == 0 and sb["device_error"] == 0

    with ClockSampler(local) as clk:
        ms = timed(lambda: step(fb, bb), args.steps, args.warmup)
    value = seg_step * args.steps * world / (ms / 1000.0) / 1e6

    pv_steps = args.per_view_steps or max(2, args.steps // 3)
    ms_pv = timed(lambda: step(fp, bp), pv_steps, 1)
    value_pv = seg_step * pv_steps * world / (ms_pv / 1000.0) / 1e6
    def fwd_step():
        new_vertices(scene)
        scene.render(step_views, B, seed, fb, out=img)

    ms_fwd = timed(fwd_step, args.steps, 2)
    value_fwd = seg_fwd * args.steps * world / (ms_fwd / 1000.0) / 1e6

    # the same step with the secondary-visibility edge term added (one edge
    # sample per camera-path vertex, picked through the edge hierarchy, two
    # side paths per accepted sample)
    bs = st.make_opts(mode="batched", use_graph=1, edge_term=edge_on | st.EDGE_TERM_SECONDARY, edge_mode=0,
                      chunk_paths=chunk, persist_blocks=persist, sec_pick="tree")
    _, ss = counts(fb, bs)
    seg_sec = seg_fwd + ss["extension_rays"] + ss["shadow_rays"]
    sec_steps = max(2, args.steps // 2)
    ms_sec = timed(lambda: step(fb, bs), sec_steps, 1)
    with_sec = {"value": round(seg_sec * sec_steps * world / (ms_sec / 1000.0) / 1e6, 3),
                "ms_per_step": round(ms_sec / sec_steps, 3), "segments_per_step": seg_sec,
                "secondary_samples_per_step": ss["secondary_samples"], "pick": "edge hierarchy"}
    if ss["secondary_samples"] == 0:
        with_sec["note"] = ("no vertex of this mesh sees a silhouette edge: the row times the pick pass and "
                            "the empty side-path passes only; with_secondary_edges_torus_knot is where it fires")
    sec_knot = None if adam else secondary_on_torus_knot(st, S, chunk, persist)

    # the same step with the optional terms and shading of the widened scope:
    # point-light shadow edges (scenes with point lights) and interpolated
    # vertex normals (a second scene created with the option)
    def step_with(scn, fopts, bopts):
        new_vertices(scn)
        scn.render(views, B, seed, fopts, out=img)
        g = (img - target) * (2 * inv_n)
        dV.zero_()
        dF.zero_()
        scn.backward(views, B, seed, g, bopts, d_vertices=dV, d_face_params=dF)

    def segments_with(scn, fopts, bopts):
        step_with(scn, fopts, bopts)
        s1 = scn.stats()
        scn.render(views, B, seed, fopts, out=img)
        s0 = scn.stats()
        assert s0["device_error"] == 0 and s1["device_error"] == 0
        return s0["extension_rays"] + s0["shadow_rays"] + s1["extension_rays"] + s1["shadow_rays"]

    widened = {}
    if not adam:
        n_w = max(2, args.steps // 2)
        if len(sc.light_pos) > 0:
            bsh = st.make_opts(mode="batched", use_graph=1, edge_term=edge_on | st.EDGE_TERM_SHADOW, edge_mode=0,
                               chunk_paths=chunk, persist_blocks=persist)
            seg_w = segments_with(scene, fb, bsh)
            ms_w = timed(lambda: step_with(scene, fb, bsh), n_w, 1)
            widened["with_shadow_edges"] = {"value": round(seg_w * n_w * world / (ms_w / 1000.0) / 1e6, 3),
                                            "ms_per_step": round(ms_w / n_w, 3), "segments_per_step": seg_w}
        import dataclasses
        sm_scene = st.Scene.from_scene(dataclasses.replace(sc, smooth_normals=True), bvh_builder=args.bvh)
        seg_w = segments_with(sm_scene, fb, bb)
        ms_w = timed(lambda: step_with(sm_scene, fb, bb), n_w, 1)
        widened["with_smooth_normals"] = {"value": round(seg_w * n_w * world / (ms_w / 1000.0) / 1e6, 3),
                                          "ms_per_step": round(ms_w / n_w, 3), "segments_per_step": seg_w}
        sm_scene.close()

    # rooflines of the two traversal kernels: algorithmic bytes from the instrumented
    # traversal (same rays), time from CUDA events around each launch
    ci = st.make_opts(mode="batched", use_graph=0, count_visits=1, chunk_paths=chunk)
    cib = st.make_opts(mode="batched", use_graph=0, count_visits=1, edge_term=edge_on, edge_mode=0, chunk_paths=chunk)
    a, b = counts(ci, cib)
    visits = a["node_visits"] + b["node_visits"]
    tests = a["tri_tests"] + b["tri_tests"]
    rays = a["extension_rays"] + b["extension_rays"]
    sh_visits = a["shadow_node_visits"] + b["shadow_node_visits"]
    sh_tests = a["shadow_tri_tests"] + b["shadow_tri_tests"]
    sh_rays = a["shadow_rays"] + b["shadow_rays"]
    ti = st.make_opts(mode="batched", use_graph=0, time_kernels=1, chunk_paths=chunk)
    tib = st.make_opts(mode="batched", use_graph=0, time_kernels=1, edge_term=edge_on, edge_mode=0, chunk_paths=chunk)
    ext_ms, ext_n, sh_ms, sh_n, reps = 0.0, 0, 0.0, 0, 3
    for _ in range(reps):
        flush.fill_(1.0)
        a, b = counts(ti, tib)
        ext_ms += a["extend_ms"] + b["extend_ms"]
        ext_n += a["extend_launches"] + b["extend_launches"]
        sh_ms += a["shadow_ms"] + b["shadow_ms"]
        sh_n += a["shadow_launches"] + b["shadow_launches"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    l2 = l2_peak_gbs(st)
    tr, tr_sh = profiled_traffic()

    def roof_record(name, v, t, q, ms, n):
        # per query: each 4-wide node fetch reads all four child boxes and links (112 B), each
        # triangle test one leaf record (48 B), plus the ray in and the hit out (48 B)
        alg = v * 112 + t * 48 + q * 48
        achieved = alg * reps / (ms / 1000.0) / 1e9
        per_launch_ms = ms / max(1, n)
        out = {"bound": "l2", "achieved": round(achieved, 2), "peak": round(l2, 1), "unit": "GB/s",
               "frac": round(achieved / l2, 4), "traffic": None, "kernel": name,
               "peak_source": "st_measure_l2_read: L2-resident read bandwidth, best of 16/32/48 MiB, measured live",
               "launch_ms_avg": round(per_launch_ms, 4), "launches_per_step": n // reps,
               "queries_per_step": q, "alg_bytes_per_query": round(alg / max(q, 1), 1),
               "node_fetches_per_query": round(v / max(q, 1), 2), "tri_tests_per_query": round(t / max(q, 1), 2),
               # the same queries counted with 64 B per node visit (a binary node), for comparison
               "alg_bytes_per_query_64B_nodes": round((v * 64 + t * 48 + q * 48) / max(q, 1), 1),
               "hbm": {"peak": hbm_peak, "unit": "GB/s",
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"}}
        return out

    roofline = roof_record("closest hit: k_raygen bin-cell tests + k_extend BVH traversal", visits, tests, rays, ext_ms,
                           ext_n)
    roofline_shadow = roof_record("k_shadow (any-hit BVH traversal)", sh_visits, sh_tests, sh_rays, sh_ms, sh_n)
    # DRAM bytes per query from the committed ncu capture (cold caches) times this step's queries per launch
    for rl, per_query, q, n in ((roofline, tr, rays, ext_n), (roofline_shadow, tr_sh, sh_rays, sh_n)):
        if per_query is None:
            continue
        per_launch = per_query * q / max(1, n // reps)
        rl["traffic"] = round(per_launch, 1)
        rl["hbm"]["dram_frac"] = round(per_launch / (rl["launch_ms_avg"] / 1000.0) / 1e9 / hbm_peak, 4)

    # where the per-view step's time goes: GPU time between its host synchronisations
    # (queue counts read back after each stage) against the step's wall time
    tp = st.make_opts(mode="per_view", use_graph=0, time_kernels=1)
    tpb = st.make_opts(mode="per_view", use_graph=0, time_kernels=1, edge_term=edge_on, edge_mode=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1.0)
    e0.record(stream)
    a, b = counts(tp, tpb)
    e1.record(stream)
    torch.cuda.synchronize()
    pv_wall = e0.elapsed_time(e1)
    pv_busy = a["busy_ms"] + b["busy_ms"]
    per_view_split = {"wall_ms": round(pv_wall, 3), "gpu_busy_ms": round(pv_busy, 3),
                      "host_sync_gap_ms": round(pv_wall - pv_busy, 3),
                      "host_syncs": a["host_syncs"] + b["host_syncs"],
                      "extend_ms": round(a["extend_ms"] + b["extend_ms"], 3),
                      "shadow_ms": round(a["shadow_ms"] + b["shadow_ms"], 3)}
    flush.fill_(1.0)
    e0.record(stream)
    a, b = counts(ti, tib)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_split = {"wall_ms": round(e0.elapsed_time(e1), 3), "gpu_busy_ms": round(a["busy_ms"] + b["busy_ms"], 3),
                     "extend_ms": round(a["extend_ms"] + b["extend_ms"], 3),
                     "shadow_ms": round(a["shadow_ms"] + b["shadow_ms"], 3), "graph": False,
                     "chunks_overlapped": False,
                     "note": "kernels timed one by one on one stream; the timed step overlaps consecutive chunks on "
                             "two engines and streams (ms_per_step)"}

    # end to end through the C ABI with host buffers: H2D of the mesh state and
    # D2H of the image and both gradients every step
    hV = torch.from_numpy(sc.vertices.copy()).pin_memory()
    hP = torch.from_numpy(sc.face_params.copy()).pin_memory()
    oI = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    oV = torch.empty((scene.nv, 3), dtype=torch.float32).pin_memory()
    oF = torch.empty(tuple(scene.face_params.shape), dtype=torch.float32).pin_memory()
    dVert = torch.empty_like(scene.vertices)
    dPar = torch.empty_like(scene.face_params)

    def e2e_step():
        if adam:
            # the model lives on the host: upload it, iterate, read the updated model back
            with torch.no_grad():
                rec.V.copy_(hV, non_blocking=True)
                rec.P.copy_(hP, non_blocking=True)
            step(fb, bb)
            oV.copy_(rec.V.detach(), non_blocking=True)
            oF.copy_(rec.P.detach(), non_blocking=True)
            return
        dVert.copy_(hV, non_blocking=True)
        dPar.copy_(hP, non_blocking=True)
        scene.refit(dVert)
        scene.set_face_params(dPar)
        step(fb, bb)
        oI.copy_(img, non_blocking=True)
        oV.copy_(dV, non_blocking=True)
        oF.copy_(dF, non_blocking=True)

    ms_e2e = timed(e2e_step, args.steps, 2)
    value_e2e = seg_step * args.steps * world / (ms_e2e / 1000.0) / 1e6
    h2d = hV.numel() * 4 + hP.numel() * 4
    d2h = (0 if adam else oI.numel() * 4) + oV.numel() * 4 + oF.numel() * 4

    # CPU-baseline leg (rank 0): the oracle timed on a pixel sample, and the same oracle
    # checking this run's launch configuration (image, signatures, gradients) on a sample
    cpu, parity = None, None
    if rank == 0 and not args.no_cpu:
        import dataclasses
        parity = oracle_parity(st, scene, dataclasses.replace(sc, views=step_views), step_target, B, seed, fb, bb,
                               edge_on)
    if rank == 0 and world == 1 and not args.no_cpu:
        r, cores, pix, secs = oracle_sample_rate(sc, args.cpu_seconds)
        r1, _, pix1, secs1 = oracle_sample_rate(sc, max(2.0, args.cpu_seconds / 4), seed=2025, threads=1)
        cpu = {"value": round(r, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d sampled pixels (all their samples): forward + interior gradient + edge term, "
                         "FP64 brute force, %.1f s" % (pix, secs),
               "single_core": {"value": round(r1, 6), "unit": UNIT, "cores": 1,
                               "sample": "%d sampled pixels, %.1f s" % (pix1, secs1)}}

    st_final = scene.stats()
    scene.close()
    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": DESCRIPTIONS[args.workload], "segments_per_step": seg_step,
                          "paths_per_step": sf["paths"] + sb["paths"], "edge_samples_per_step": sb["edge_samples"],
                          "l2": "flushed between timed steps (256 MiB write)", "launch": "batched persistent + CUDA graph",
                          "autotuned": None if tuned is None else {k: tuned[k] for k in ("chunk_paths", "persist_blocks")},
                          "edge_term": bool(edge_on), "bvh": args.bvh,
                          "scene_create_ms": round(1000 * t_build, 1),
                          "parallelism": "replicas" if world > 1 else "single GPU"},
               "batched_vs_per_view": round(value / value_pv, 3),
               "per_view": {"value": round(value_pv, 3), "ms_per_step": round(ms_pv / pv_steps, 3),
                            "launch": "per-view, host-read queue counts, no graph"},
               "forward_only": {"value": round(value_fwd, 3), "ms_per_step": round(ms_fwd / args.steps, 3)},
               "with_secondary_edges": with_sec, "with_secondary_edges_torus_knot": sec_knot, **widened,
               "roofline": roofline, "roofline_k_shadow": roofline_shadow,
               "time_split": {"per_view": per_view_split, "batched_ungraphed": batched_split},
               "grad_rel_err": None if parity is None else parity["grad_rel_err"], "parity": parity,
               "cpu_baseline": cpu,
               "e2e": {"value": round(value_e2e, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e / args.steps, 3)},
               "gpu_launches": launches_step * args.steps, "clocks": clk.summary(),
               "device_error": st_final["device_error"]}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
