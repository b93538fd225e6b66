"""Benchmark: tiles/s of the display-driven tile renderer on one GB300.

Workload (default): 100M clustered points (64-component Gaussian mixture +
5% uniform noise, int32 grid), 10,000 density-weighted tiles at zoom 8-14,
radius 2 px, RGBA output (HiVision Exp. 2 shape: 10,000 random tiles, no
result cache).  A step renders the whole batch of tiles with one call of
hv_render_tiles (device-resident requests and output).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun): every rank holds a replica of the layer and renders the
tiles the tile router (hv_route_tiles) sends it out of a batch of N x 10,000
(weak scaling, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import gen  # noqa: E402

WORKLOADS = {
    2: {"workload": "clustered points 100M (64-Gaussian mixture + 5% noise, int32 grid), "
                    "10,000 density-weighted 256x256 tiles at zoom 8-14, radius 2 px, RGBA",
        "n_objects": 100_000_000, "tiles_per_step": 10_000, "zoom": [8, 14], "r16": 32, "mode": "rgba"},
    3: {"workload": "random-walk linestrings 50M segments in 5M lines around 1,000 city centres "
                    "(int32 grid), 10,000 density-weighted tiles at zoom 6-16, half-width 1 px, RGBA",
        "n_objects": 50_000_000, "n_lines": 5_000_000, "tiles_per_step": 10_000, "zoom": [6, 16],
        "r16": 16, "mode": "rgba"},
    4: {"workload": "star polygons 2M (8-64 vertices, 256-Gaussian mixture centres, int32 grid), "
                    "10,000 density-weighted tiles at zoom 4-14, fill + 1 px outline, RGBA",
        "n_objects": 2_000_000, "tiles_per_step": 10_000, "zoom": [4, 14], "r16": 8, "mode": "rgba"},
}
WORKLOAD = WORKLOADS[2]
METRIC = "tiles/sec (256² px) and p99 tile latency, learned vs R-tree index, 1 GB300"
STYLE_T = (230, 40, 20, 0, 30, 90, 200, 0)
NOUN = {"points": "points", "lines": "segments", "polygons": "polygons"}
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 4, 5],
                    help="2: clustered points (the headline), 3: linestrings, 4: polygons, "
                         "5: serving an open-loop request stream over resident layers")
    ap.add_argument("--rates", default="5000,10000,20000,50000,inf",
                    help="config 5: request rates (tiles/s), 'inf' = all at once")
    ap.add_argument("--requests", type=int, default=100_000, help="config 5: requests per rate")
    ap.add_argument("--serve-points", type=int, default=1_000_000_000)
    ap.add_argument("--serve-segments", type=int, default=200_000_000)
    ap.add_argument("--r16", type=int, default=None)
    ap.add_argument("--points", type=int, default=None, help="objects (points / segments / polygons)")
    ap.add_argument("--tiles", type=int, default=WORKLOAD["tiles_per_step"])
    ap.add_argument("--cpu-sample-tiles", type=int, default=None,
                    help="oracle sample (default 48 / 16 / 6 tiles for configs 2 / 3 / 4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--count-sample-tiles", type=int, default=200)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--index", default="rtree", choices=["rtree", "learned"],
                    help="index timed for the headline value (both are reported)")
    ap.add_argument("--no-host-placement", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the clustered-points line, without the blocks of the other workloads")
    ap.add_argument("--profile-steps", action="store_true",
                    help="only warm-up + steps, no baselines (for ncu launch lists)")
    ap.add_argument("--volume-sweep", default=None,
                    help="comma-separated point counts: the clustered-points tiles rendered over layers of "
                         "each size (the same 10,000 tiles), one JSON line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples nvidia-smi every 200 ms while running (start/stop around the
    timed region)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("hv_render.cu", "hv_device.cuh", "hv_learned.cuh", "hv_internal.h")
PROFILES = {2: "k_render_points_gmm100M.md", 3: "k_render_lines_walk50M.md", 4: "k_render_polygons_star2M.md"}


def _code_only(text):
    """Source text without // and /* */ comments and without whitespace (the
    files hashed below hold no string literal with comment markers)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r"\s+", "", text)


def kernel_source_hash():
    """sha256 over the code (comments and whitespace removed) of the sources
    the render kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2005_12489_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def _profile_record(cfg, key):
    """The integer recorded under `key` in the committed ncu summary of the
    workload's render kernel, if the kernel code still hashes to the value
    recorded beside it; else None."""
    path = os.path.join(ROOT, "profiles", PROFILES.get(cfg, ""))
    if not os.path.isfile(path):
        return None
    want = kernel_source_hash()
    for ln in open(path):
        if ln.startswith(key + ":"):
            parts = ln.split()
            if len(parts) >= 4 and parts[2] == "kernel_sources_sha256" and parts[3] == want:
                return int(parts[1])
    return None


def measured_instructions(cfg):
    """Warp instructions one full-size launch (both launches of a polygon step)
    executes, from the committed ncu summary (None once the kernel changed)."""
    return _profile_record(cfg, "instructions_per_launch")


def issue_peak():
    """Issue-rate ceiling in G warp instructions/s: SMs x 4 schedulers x one
    warp instruction per cycle at the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return sms * 4 * mhz * 1e6 / 1e9


def measured_traffic(cfg):
    """DRAM bytes (read + write) of one full-size launch of the render kernel,
    from the committed ncu summary, if the kernel sources still hash to the
    value recorded beside it; else None."""
    return _profile_record(cfg, "traffic_per_launch_bytes")


class Layer:
    """A workload's layer as host arrays, with loaders for the library and the oracle."""

    def __init__(self, cfg, args, rank):
        w = WORKLOADS[cfg]
        self.cfg = cfg
        n = args.points or w["n_objects"]
        r16 = args.r16 or w["r16"]
        z0, z1 = w["zoom"]
        # every rank renders its own args.tiles tiles: shard `rank` of a batch
        # of args.tiles * world requests (weak scaling over replicas)
        world = dist_env()[1]
        if cfg == 2:
            self.kind = "points"
            self.xy = gen.gmm_points(n, seed=2, k=64)
            all_reqs = gen.density_tiles(self.xy, args.tiles * world, z0, z1, r16, seed=102)
            self.obj_bytes = 8
        elif cfg == 3:
            self.kind = "lines"
            n_lines = max(1, n // 10)
            self.xy, self.off = gen.walk_lines(n_lines, n, seed=3)
            mids = gen.segment_midpoints(self.xy, self.off, max_n=4 * args.tiles, seed=103)
            all_reqs = gen.density_tiles(mids, args.tiles * world, z0, z1, r16, seed=203)
            self.obj_bytes = 32      # index record: segment + piece box
        else:
            self.kind = "polygons"
            self.xy, self.ro, self.po = gen.star_polygons(n, seed=4)
            cen = gen.polygon_centres(self.xy, self.ro, self.po)
            all_reqs = gen.density_tiles(cen, args.tiles * world, z0, z1, r16, seed=104)
            self.obj_bytes = 32      # index record: edge + piece box
            ro = np.asarray(self.ro, dtype=np.int64)
            po = np.asarray(self.po, dtype=np.int64)
            self.poly_edges = ro[po[1:]] - ro[po[:-1]]
        if world > 1:
            # replicas: the tile router sends each tile to one rank
            from paper_2005_12489_gb300 import hv
            self.reqs = all_reqs[hv.hv_route_tiles(all_reqs, world) == rank]
        else:
            self.reqs = all_reqs
        self.n_objects = n

    def load(self, hv, ctx):
        if self.kind == "points":
            return hv.hv_layer_load_points(ctx, self.xy)
        if self.kind == "lines":
            return hv.hv_layer_load_linestrings(ctx, self.xy, self.off)
        return hv.hv_layer_load_polygons(ctx, self.xy, self.ro, self.po)

    def oracle(self, reqs, mode=2):
        import oracle
        oracle.build()
        if self.kind == "points":
            return oracle.render_points(self.xy, reqs, mode, STYLE_T)
        if self.kind == "lines":
            return oracle.render_lines(self.xy, self.off, reqs, mode, STYLE_T)
        return oracle.render_polygons(self.xy, self.ro, self.po, reqs, mode, STYLE_T)


def workload(args, rank):
    return Layer(args.config, args, rank)


def cpu_baseline(lay, n_sample):
    """The oracle (single-threaded C, data driven) on a bounded sample of the
    batch's tiles: one pass over all objects for n_sample tiles."""
    reqs = lay.reqs
    sample = reqs[np.linspace(0, len(reqs) - 1, n_sample).astype(np.int64)]
    t0 = time.perf_counter()
    lay.oracle(sample)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": "tiles/s", "cores": 1, "kind": "oracle",
            "sample": "%d of the %d tiles (evenly spaced), all %d %s, single-threaded C"
                      % (n_sample, len(reqs), lay.n_objects, NOUN[lay.kind]), "seconds": dt}


def cpu_rtree_baseline(lay, n_sample):
    """The multithreaded CPU R-tree renderer (the paper's pixel-driven method
    with the exact per-sample rule) on all host cores, on an evenly spaced
    sample of the batch."""
    import cpu_baseline
    t0 = time.perf_counter()
    if lay.kind == "points":
        tree = cpu_baseline.PointTree(lay.xy)
    elif lay.kind == "lines":
        tree = cpu_baseline.LineTree(lay.xy, lay.off)
    else:
        tree = cpu_baseline.PolygonTree(lay.xy, lay.ro, lay.po)
    build_s = time.perf_counter() - t0
    sample = lay.reqs[np.linspace(0, len(lay.reqs) - 1, n_sample).astype(np.int64)]
    t0 = time.perf_counter()
    _, threads = tree.render(sample, STYLE_T)
    dt = time.perf_counter() - t0
    tree.close()
    return {"value": n_sample / dt, "unit": "tiles/s", "cores": threads,
            "kind": "cpu packed R-tree, per-sample queries",
            "sample": "%d of the %d tiles (evenly spaced), all %d %s" % (n_sample, len(lay.reqs), lay.n_objects,
                                                                        NOUN[lay.kind]),
            "build_s": build_s, "seconds": dt}


def run_reference(args):
    """The oracle as the reference arm, on the host cores (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    lay = workload(args, 0)
    reqs = lay.reqs
    n_sample = 8
    times = []
    for step in range(args.warmup + args.steps):
        sample = reqs[(np.arange(n_sample) * 997 + step * 13) % len(reqs)]
        t0 = time.perf_counter()
        lay.oracle(sample)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    value = n_sample * len(times) / sum(times)
    # n_gpus: the launch's N (this arm itself runs on one host core)
    line = {"metric": METRIC, "value": value, "unit": "tiles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference",
            "config": dict(WORKLOADS[args.config], n_objects=lay.n_objects, sample_tiles_per_step=n_sample),
            "cpu_baseline": {"value": value, "unit": "tiles/s", "cores": 1, "kind": "oracle",
                             "sample": "%d tiles per step of the %d-tile batch, all %d %s"
                                       % (n_sample, len(reqs), lay.n_objects, NOUN[lay.kind])},
            "e2e": {"value": value, "unit": "tiles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def algorithmic_bytes_per_tile(hv, layer, reqs_dev_np, torch, n_sample, lay):
    """Unique bytes the early-exit traversal must read per tile (inner nodes x
    512 B + visited leaves x 32 objects x object size, polygon boxes and the
    edges of the polygons whose parity was evaluated) plus the tile's output
    and its request, from the library's instrumented visit log on a tile
    sample; non-unique visit counts are reported beside it."""
    idx = np.linspace(0, len(reqs_dev_np) - 1, n_sample).astype(np.int64)
    sample = reqs_dev_np[idx]
    log = torch.empty(1 << 27, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_req = torch.from_numpy(hv.make_requests(sample).view(np.uint8).copy()).cuda()
    out = torch.empty((len(sample), hv.hv_tile_bytes(hv.HV_MODE_RGBA)), dtype=torch.uint8, device="cuda")
    hv.hv_render_tiles_counted(layer, d_req, len(sample), hv.HV_MODE_RGBA, hv.HV_INDEX_RTREE,
                               hv.make_style(), out, out.numel(), log, log.numel(), cnt)
    torch.cuda.synchronize()
    n = int(cnt.item())
    if n > log.numel():
        return None
    visits = log[:n]
    vkind = (visits >> 35) & 7
    keys = torch.unique(visits)
    kind = (keys >> 35) & 7
    nodes = int((kind == 0).sum().item())
    leaves = int((kind == 1).sum().item())
    pnodes = int((kind == 2).sum().item())
    pleaves = int((kind == 3).sum().item())
    read = nodes * 512 + leaves * 32 * lay.obj_bytes + pnodes * 512 + pleaves * 32 * 20
    if lay.kind == "polygons":
        pid = (keys[kind == 4] & ((1 << 35) - 1)).cpu().numpy()
        read += int(lay.poly_edges[pid].sum()) * 16 + 16 * len(pid)
    k = len(sample)
    per_tile = read / k + hv.hv_tile_bytes(hv.HV_MODE_RGBA) + 16
    node_visits = int(((vkind == 0) | (vkind == 2)).sum()) / k
    leaf_visits = int(((vkind == 1) | (vkind == 3)).sum()) / k
    return {"per_tile": per_tile, "read_per_tile": read / k, "unique_nodes_per_tile": (nodes + pnodes) / k,
            "unique_leaves_per_tile": (leaves + pleaves) / k, "node_visits_per_tile": node_visits,
            "leaf_visits_per_tile": leaf_visits, "node_visits_per_pixel": node_visits / 65536,
            "leaf_visits_per_pixel": leaf_visits / 65536, "sample_tiles": k}


def _timed(step, flush, stream, k_steps, warm=2):
    """Mean device time (ms) of k_steps calls of step(), each bracketed by CUDA
    events on `stream`, the L2 flushed before each."""
    import torch
    for _ in range(warm):
        flush.fill_(1)
        step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
    for k in range(k_steps):
        flush.fill_(k & 255)
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _latency(hv, torch, layer, d_req, n, mode, index, style, stream, n_tiles=300):
    """Per-tile latency: batch-1 calls, each timed with CUDA events."""
    tb = hv.hv_tile_bytes(mode)
    idx = np.linspace(0, n - 1, n_tiles).astype(np.int64)
    one = torch.empty((1, tb), dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_tiles)]
    req_rows = d_req.view(n, 16)
    for k, t in enumerate(idx):
        evs[k][0].record(stream)
        hv.hv_render_tiles(layer, req_rows[int(t)], 1, mode, index, style, one, one.numel(), stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) for a, b in evs])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "tiles": n_tiles, "form": "batch-1 calls, device buffers"}


def phase_profile(hv, torch, layer, d_req, n, mode, index, style, d_out, kind):
    """Where the render kernel's time goes: one launch of the instrumented
    instantiation (hv_render_tiles_phases), as shares of the launch's
    warp-cycles, and visit counts per tile.  Polygon layers report the outline
    and the fill launch apart."""
    cnt = hv.HV_PHASE_COUNT * (2 if kind == "polygons" else 1)
    ph = torch.zeros(cnt, dtype=torch.int64, device="cuda")
    hv.hv_render_tiles_phases(layer, d_req, n, mode, index, style, d_out, d_out.numel(), ph)
    torch.cuda.synchronize()
    v = ph.cpu().numpy().astype(np.float64)
    parts = {}
    for k, name in enumerate(["fill", "outline"] if kind == "polygons" else ["render"]):
        c = v[hv.HV_PHASE_COUNT * k:hv.HV_PHASE_COUNT * (k + 1)]
        tot = max(c[0], 1.0)
        busy, leaf, desc = c[5], c[6], c[7]
        parts[name] = {
            "share": {"prologue": c[1] / tot, "cull": c[2] / tot, "bin": c[3] / tot,
                      "frontier_scan": (busy - desc) / tot, "node_tests": (desc - leaf) / tot,
                      "leaf_visits": leaf / tot, "blocks_waiting": (c[4] - busy) / tot, "encode": c[8] / tot},
            "per_tile": {"blocks": c[10] / n, "leaf_visits": c[11] / n, "node_visits": c[12] / n,
                         "frontier_tests": c[13] / n, "leaf_visits_empty": c[14] / n,
                         "leaf_visits_deciding": c[15] / n},
            "warp_cycles_per_tile": tot / n}
    return parts


def _learned_info(info):
    return {"error_bound": info.learned_error, "error_bound_linear": info.learned_error_linear,
            "error_bound_mlp": info.learned_error_mlp, "mean_error": info.learned_mean_error,
            "pieces": info.learned_pieces, "pieces_with_mlp": info.learned_mlp,
            "mean_window": info.learned_mean_window, "mean_window_linear": info.learned_mean_window_linear,
            "halo": info.learned_halo, "side_tree_objects": info.learned_outliers, "train_ms": info.train_ms}


def _roofline(alg, n, ms, cfg, full_size, launch_ms=None):
    """HBM roofline of the render kernel(s): algorithmic bytes per launch over
    the launch time (the step's device time: one call is one launch, two for
    polygon layers)."""
    if alg is None:
        return None
    peak, peak_kind = measured_peak_hbm()
    achieved = alg["per_tile"] * n / (ms / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic(cfg) if full_size else None, "peak_kind": peak_kind,
            "kernel": "k_render", "alg_bytes_per_tile": alg["per_tile"], "alg_detail": alg}


def _roofline_issue(cfg, ms, full_size):
    n_inst = measured_instructions(cfg) if full_size else None
    if n_inst is None:
        return None
    ipk = issue_peak()
    achieved_i = n_inst / (ms / 1000.0) / 1e9
    return {"bound": "alu", "achieved": achieved_i, "peak": ipk, "unit": "G warp-instructions/s",
            "frac": achieved_i / ipk, "instructions_per_launch": n_inst,
            "peak_basis": "SMs x 4 schedulers x 1 warp instruction/cycle x max SM clock",
            "note": "the integer pipe bounds this kernel; instruction count from the committed ncu summary"}


def measure_batch(args, cfg, steps, warmup, dist=None, headline=False, r16_sweep=None):
    """One batch workload (clustered points, linestrings or polygons): a step
    renders the whole batch of tiles with one hv_render_tiles call (device
    requests and output).  Returns the JSON dict of the workload; with
    `headline` the timed region follows the full contract (barrier, clocks,
    max over ranks) and extras run on rank 0 only."""
    import torch
    from paper_2005_12489_gb300 import hv

    rank, world, local = dist_env()
    w = WORKLOADS[cfg]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    a = argparse.Namespace(**vars(args))
    if not headline:
        a.points, a.r16, a.tiles = None, None, w["tiles_per_step"]
    lay = Layer(cfg, a, rank)
    reqs = lay.reqs
    ctx = hv.hv_create(local)
    layer = lay.load(hv, ctx)
    want_learned = (not args.no_learned) or args.index == "learned"
    hv.hv_layer_build_index(layer, hv.HV_INDEX_RTREE | (hv.HV_INDEX_LEARNED if want_learned else 0))
    info = hv.hv_layer_info_get(layer)
    main_index = hv.HV_INDEX_LEARNED if (headline and args.index == "learned") else hv.HV_INDEX_RTREE
    mode = hv.HV_MODE_RGBA
    tb = hv.hv_tile_bytes(mode)
    n = len(reqs)
    style = hv.make_style(STYLE_T[:3], STYLE_T[4:7])
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    d_out = torch.empty((n, tb), dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    launches_per_step = hv.hv_render_launches(layer, main_index)

    def step(index=main_index, reqs_dev=d_req):
        hv.hv_render_tiles(layer, reqs_dev, n, mode, index, style, d_out, d_out.numel(), stream)

    for _ in range(warmup):
        flush.fill_(1)
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = Clocks(local)
    barrier()
    clocks.start()
    t0 = time.perf_counter()
    for k in range(steps):
        flush.fill_(k & 255)            # L2 flush between steps (not timed)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    step_ms = [x.elapsed_time(y) for x, y in ev]
    ms = sum(step_ms) / len(step_ms)
    total = n
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        tn = torch.tensor([n], dtype=torch.int64, device="cuda")
        dist.all_reduce(tn, op=dist.ReduceOp.SUM)
        total = int(tn.item())
    value = total / (ms / 1000.0)
    out = None
    if rank == 0 and not args.profile_steps:
        lat = {"rtree": _latency(hv, torch, layer, d_req, n, mode, hv.HV_INDEX_RTREE, style, stream)}
        learned = None
        k_side = max(3, min(steps, 10))
        if want_learned:
            info = hv.hv_layer_info_get(layer)
            lms = statistics.mean(_timed(lambda: step(hv.HV_INDEX_LEARNED), flush, stream, k_side))
            rms = ms if main_index == hv.HV_INDEX_RTREE else statistics.mean(
                _timed(lambda: step(hv.HV_INDEX_RTREE), flush, stream, k_side))
            lat["learned"] = _latency(hv, torch, layer, d_req, n, mode, hv.HV_INDEX_LEARNED, style, stream)
            learned = dict({"value": n / (lms / 1000.0), "ms_per_step": lms, "unit": "tiles/s",
                            "rtree_value": n / (rms / 1000.0), "learned_over_rtree": rms / lms},
                           **_learned_info(info))
        sweep = None
        if r16_sweep:
            sweep = []
            for r16 in r16_sweep:
                rr = reqs.copy()
                rr[:, 3] = r16
                d2 = torch.from_numpy(hv.make_requests(rr).view(np.uint8).copy()).cuda()
                row = {"r16": r16, "half_width_px": r16 / 16.0}
                rt = statistics.mean(_timed(lambda: step(hv.HV_INDEX_RTREE, d2), flush, stream, k_side))
                row["rtree_tiles_per_s"] = n / (rt / 1000.0)
                if want_learned:
                    le = statistics.mean(_timed(lambda: step(hv.HV_INDEX_LEARNED, d2), flush, stream, k_side))
                    row["learned_tiles_per_s"] = n / (le / 1000.0)
                    row["learned_over_rtree"] = rt / le
                sweep.append(row)
        phases = {"rtree": phase_profile(hv, torch, layer, d_req, n, mode, hv.HV_INDEX_RTREE, style, d_out, lay.kind)}
        if want_learned:
            phases["learned"] = phase_profile(hv, torch, layer, d_req, n, mode, hv.HV_INDEX_LEARNED, style, d_out,
                                              lay.kind)
        placed = None
        if headline and not args.no_host_placement:
            # the same layer with its index records in host memory, read over
            # the CPU-GPU link (NVLink-C2C): what a layer larger than the
            # device's memory would run at
            hl = lay.load(hv, ctx)
            opts = hv.hv_build_opts()
            opts.object_placement = hv.HV_PLACE_HOST
            hv.hv_layer_build_index(hl, hv.HV_INDEX_RTREE, opts)
            hinfo = hv.hv_layer_info_get(hl)

            def hstep():
                hv.hv_render_tiles(hl, d_req, n, mode, hv.HV_INDEX_RTREE, style, d_out, d_out.numel(), stream)
            hms = statistics.mean(_timed(hstep, flush, stream, k_side))
            placed = {"value": n / (hms / 1000.0), "unit": "tiles/s", "ms_per_step": hms,
                      "over_device_resident": ms / hms, "host_bytes": hinfo.host_bytes,
                      "device_bytes": hinfo.device_bytes,
                      "placement": "index records in pinned host memory (mapped), nodes and keys in HBM"}
            hv.hv_layer_free(hl)
        full_size = (args.points is None and args.r16 is None and n == w["tiles_per_step"]) or not headline
        alg = algorithmic_bytes_per_tile(hv, layer, reqs, torch, args.count_sample_tiles, lay)
        roof = _roofline(alg, n, ms, cfg, full_size)
        roof_issue = _roofline_issue(cfg, ms, full_size)
        e2e = None
        if not args.no_e2e:
            h_req = hv.make_requests(reqs)
            h_out = torch.empty((n, tb), dtype=torch.uint8, pin_memory=True)
            for _ in range(2):
                hv.hv_render_tiles(layer, h_req, n, mode, main_index, style, h_out, h_out.numel(), stream)
            k_e2e = max(3, min(steps, 10))
            t1 = time.perf_counter()
            for _ in range(k_e2e):
                hv.hv_render_tiles(layer, h_req, n, mode, main_index, style, h_out, h_out.numel(), stream)
            dt = (time.perf_counter() - t1) / k_e2e
            # the copy bound: a plain pinned device -> host copy of 1 GiB
            cb = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
            hb = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
            hb.copy_(cb)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            for _ in range(3):
                hb.copy_(cb)
            torch.cuda.synchronize()
            d2h = 3 * (1 << 30) / (time.perf_counter() - t2) / 1e9
            del cb, hb
            e2e = {"value": n / dt, "unit": "tiles/s", "h2d_bytes_per_step": int(h_req.nbytes),
                   "d2h_bytes_per_step": int(n * tb), "ms_per_step": 1000 * dt,
                   "over_device": (n / dt) / (n / (ms / 1000.0)), "d2h_copy_GBps": d2h,
                   "copy_bound_ms": n * tb / d2h / 1e6,
                   "path": "hv_render_tiles with host requests and pinned host output (the kernels write the "
                           "tiles into it over the CPU-GPU link)"}
        n_cpu = args.cpu_sample_tiles or {2: 48, 3: 8, 4: 4}[cfg]
        cpu = None if args.no_cpu_baseline else cpu_baseline(lay, n_cpu)
        cpu_mt = None if args.no_cpu_baseline else cpu_rtree_baseline(lay, {2: 96, 3: 48, 4: 16}[cfg])
        out = {"metric": METRIC, "value": value, "unit": "tiles/s", "n_gpus": world,
               "steps": steps, "warmup": warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
               "data": "synthetic",
               "config": dict(w, index="packed Hilbert R-tree" if main_index == hv.HV_INDEX_RTREE else "learned",
                              n_objects=lay.n_objects, tiles_per_step=n,
                              r16=int(reqs[0, 3]) if n else w["r16"],
                              l2="flushed between steps (512 MiB write); layer and output exceed L2",
                              parallelism="replicas" if world > 1 else "single GPU"),
               "pixel_queries_per_s": value * 65536,
               "roofline": roof, "roofline_issue": roof_issue, "cpu_baseline": cpu, "cpu_rtree_mt": cpu_mt,
               "e2e": e2e, "gpu_launches": launches_per_step * steps, "clocks": clk,
               "index_timed": "rtree" if main_index == hv.HV_INDEX_RTREE else "learned",
               "learned": learned, "latency": lat, "r16_sweep": sweep, "phases": phases,
               "host_resident": placed,
               "wall_s_timed_region": wall, "step_ms": step_ms,
               "index_build_ms": info.build_ms, "tree_levels": info.tree_levels,
               "index_records": info.index_records, "piece_extent": info.piece_extent}
    elif rank == 0:
        out = {"profile_steps": True, "ms_per_step": ms}
    del d_out, flush
    hv.hv_layer_free(layer)
    hv.hv_destroy(ctx)
    return out


def run_gb300(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    line = measure_batch(args, args.config, args.steps, args.warmup, dist, headline=True,
                         r16_sweep=(8, 16, 24) if args.config == 3 else None)
    if rank == 0 and line is not None and not args.profile_steps and world == 1 and not args.headline_only \
            and args.config == 2:
        # the metric's other workloads, as named blocks of the same line: the
        # linestring and polygon batches (learned vs R-tree) and the served
        # request stream (p50 / p99 per rate, learned vs R-tree)
        blocks = {}
        for cfg in (3, 4):
            t0 = time.time()
            blocks[str(cfg)] = measure_batch(args, cfg, 5, 3, None, headline=False,
                                             r16_sweep=(8, 16, 24) if cfg == 3 else None)
            blocks[str(cfg)]["wall_s"] = time.time() - t0
            print("config %d done in %.0f s" % (cfg, time.time() - t0), file=sys.stderr, flush=True)
        t0 = time.time()
        blocks["5"] = serving_block(args)
        blocks["5"]["wall_s"] = time.time() - t0
        line["configs"] = blocks
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def _serve_rate(hv, ctx, layers, reqs, arrival, index, style, max_batch=64):
    """Replay one request stream through a fresh server; per-request
    submit-to-completion latency and its parts from the server's own
    timestamps (queue: submit -> batch launch; service: launch -> completion
    seen by the worker; handout: completion -> poll)."""
    opts = hv.make_server_opts(max_batch=max_batch, queue_capacity=1 << 20, scratch_bytes=4 << 30,
                               index_kind=index, use_graphs=1, style=style)
    srv = hv.hv_server_start(ctx, layers, opts)
    try:
        lat, parts, wall = hv.hv_server_replay_detail(srv, reqs, arrival)
        st = hv.hv_server_stats(srv)
    finally:
        hv.hv_server_stop(srv)
    return lat, parts, wall, st


def _latency_parts(lat, parts):
    """p50 / p99 of each part of the served latency, and the mean parts of
    the requests at or above the p99 latency (what the tail is made of)."""
    names = ("pre_submit", "task_pool", "service", "handout")
    tail = lat >= np.percentile(lat, 99)
    out = {}
    for k, nm in enumerate(names):
        out[nm] = {"p50_ms": float(np.percentile(parts[:, k], 50)) / 1000,
                   "p99_ms": float(np.percentile(parts[:, k], 99)) / 1000,
                   "tail_mean_ms": float(parts[tail, k].mean()) / 1000}
    return out


def serving_block(args):
    """Open-loop serving over resident layers (HiVision Exp. 3 shape, Sec. 5.3):
    1B clustered points + 200M random-walk segments, requests from pan/zoom
    sessions (Zipf start tiles, mixed zoom 2-18, layer 50/50, r16 16-48,
    RGBA), Poisson arrivals at each rate; per rate and index: achieved tiles/s
    and p50/p99 latency (completion - scheduled arrival, through the server's
    public calls)."""
    import torch
    from paper_2005_12489_gb300 import hv
    _, _, local = dist_env()
    t0 = time.time()
    pts = gen.gmm_points(args.serve_points, seed=5, k=64)
    n_lines = max(1, args.serve_segments // 10)
    xy, off = gen.walk_lines(n_lines, args.serve_segments, seed=55)
    gen_s = time.time() - t0
    ctx = hv.hv_create(local)
    layers = [hv.hv_layer_load_points(ctx, pts), hv.hv_layer_load_linestrings(ctx, xy, off)]
    t1 = time.time()
    for L in layers:
        hv.hv_layer_build_index(L, hv.HV_INDEX_RTREE | hv.HV_INDEX_LEARNED)
    build_s = time.time() - t1
    anchors = [pts[:: max(1, len(pts) // 2_000_000)], gen.segment_midpoints(xy, off, 2_000_000, seed=56)]
    style = hv.make_style(STYLE_T[:3], STYLE_T[4:7])
    results = []
    rates = args.rates.split(",")
    tr0 = None
    for ri, rate in enumerate(rates):
        tr = gen.pan_zoom_trace(anchors, args.requests, seed=500 + ri)
        if tr0 is None:
            tr0 = tr
        reqs = np.zeros(len(tr), dtype=hv.REQ_DTYPE)
        reqs["z"], reqs["x"], reqs["y"], reqs["r16"], reqs["layer"] = tr[:, 0], tr[:, 1], tr[:, 2], tr[:, 3], tr[:, 4]
        reqs["mode"] = hv.HV_MODE_RGBA
        arrival = np.zeros(len(reqs)) if rate == "inf" else gen.poisson_arrivals(len(reqs), float(rate), seed=600 + ri)
        for index in (hv.HV_INDEX_LEARNED, hv.HV_INDEX_RTREE):
            lat, parts, wall, st = _serve_rate(hv, ctx, layers, reqs, arrival, index, style)
            results.append({"rate": rate, "index": "learned" if index == hv.HV_INDEX_LEARNED else "rtree",
                            "requests": len(reqs), "tiles_per_s": len(reqs) / (wall / 1e6),
                            "p50_ms": float(np.percentile(lat, 50)) / 1000,
                            "p99_ms": float(np.percentile(lat, 99)) / 1000,
                            "parts": _latency_parts(lat, parts),
                            "mean_batch": st["tiles"] / max(1, st["batches"]), "slots": st["slots"],
                            "graph_launches": st["graph_launches"]})
            print(json.dumps(results[-1]), file=sys.stderr, flush=True)
    # the served kernels on the device: the first trace's requests rendered
    # per layer in batches of 64 (the server's batch) with CUDA events
    stream = torch.cuda.current_stream()
    dev = {}
    tb = hv.hv_tile_bytes(hv.HV_MODE_RGBA)
    d_out = torch.empty((64, tb), dtype=torch.uint8, device="cuda")
    for li, name in ((0, "points"), (1, "lines")):
        sel = tr0[tr0[:, 4] == li][:, :4][:4096]
        d_req = torch.from_numpy(hv.make_requests(sel).view(np.uint8).copy()).cuda()
        row = {}
        for index, iname in ((hv.HV_INDEX_RTREE, "rtree"), (hv.HV_INDEX_LEARNED, "learned")):
            def go():
                for b in range(0, len(sel), 64):
                    k = min(64, len(sel) - b)
                    hv.hv_render_tiles(layers[li], d_req[b * 16:(b + k) * 16], k, hv.HV_MODE_RGBA, index, style,
                                       d_out, d_out.numel(), stream)
            ms = statistics.mean(_timed(go, torch.empty(8, dtype=torch.uint8, device="cuda"), stream, 3, 1))
            row[iname + "_tiles_per_s"] = len(sel) / (ms / 1000.0)
        class _L:
            kind = name
            obj_bytes = 8 if li == 0 else 32
        # one tile at a time (device time of a served request's kernels)
        row["batch1"] = _latency(hv, torch, layers[li], d_req, len(sel), hv.HV_MODE_RGBA, hv.HV_INDEX_LEARNED,
                                 style, stream, n_tiles=500)
        alg = algorithmic_bytes_per_tile(hv, layers[li], sel, torch, min(200, len(sel)), _L)
        row["alg_bytes_per_tile"] = alg and alg["per_tile"]
        row["hbm_GBps"] = alg and alg["per_tile"] * row["rtree_tiles_per_s"] / 1e9
        row["tiles"] = len(sel)
        dev[name] = row
    infos = [hv.info_dict(L) for L in layers]
    for L in layers:
        hv.hv_layer_free(L)
    hv.hv_destroy(ctx)
    peak, peak_kind = measured_peak_hbm()
    # the dominant served kernel: the point layer's (its tiles are the heavier)
    hb = dev["points"]["hbm_GBps"]
    roof = None if hb is None else {"bound": "hbm", "achieved": hb, "peak": peak, "unit": "GB/s",
                                    "frac": hb / peak, "traffic": None, "peak_kind": peak_kind,
                                    "kernel": "k_render (points, batches of 64 trace tiles)",
                                    "alg_bytes_per_tile": dev["points"]["alg_bytes_per_tile"]}
    # the oracle on one trace tile of each layer over the whole layers
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t2 = time.perf_counter()
        for li in (0, 1):
            one = tr0[tr0[:, 4] == li][:1, :4].astype(np.uint32)
            if li == 0:
                oracle.render_points(pts, one, 2, STYLE_T)
            else:
                oracle.render_lines(xy, off, one, 2, STYLE_T)
        dt = time.perf_counter() - t2
        cpu = {"value": 2 / dt, "unit": "tiles/s", "cores": 1, "kind": "oracle", "seconds": dt,
               "sample": "one trace tile of each layer over all %d points + %d segments, single-threaded C"
                         % (args.serve_points, args.serve_segments)}
    del pts, xy, off
    inf_l = [r for r in results if r["rate"] == "inf" and r["index"] == "learned"]
    best = max(r["tiles_per_s"] for r in results if r["index"] == "learned")
    e2e = {"value": (inf_l[0] if inf_l else max(results, key=lambda r: r["tiles_per_s"]))["tiles_per_s"],
           "unit": "tiles/s", "h2d_bytes_per_step": 16, "d2h_bytes_per_step": tb,
           "path": "hv_server_submit / hv_server_poll, all requests offered at once; a step is one request "
                   "(host request in, RGBA tile out to pinned host memory)"}
    return {"metric": "served tiles/s and p50/p99 tile latency, open-loop request stream, learned vs R-tree",
            "value": best, "unit": "tiles/s", "higher_is_better": True,
            "config": {"workload": "resident layers: %d clustered points + %d random-walk segments; "
                                   "pan/zoom session requests (Zipf start tiles, zoom 2-18, layer 50/50, "
                                   "r16 16-48, RGBA), Poisson arrivals" % (args.serve_points, args.serve_segments),
                       "requests_per_rate": args.requests, "max_batch": 64, "graphs": True},
            "per_rate": results, "device": dev, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "generate_s": gen_s, "index_build_s": build_s,
            "layers": [{k: v for k, v in i.items() if k in ("n_objects", "learned_error", "learned_outliers",
                                                           "train_ms", "build_ms", "device_bytes")}
                       for i in infos]}


def run_serving(args):
    """--config 5 alone: the serving block as its own JSON line."""
    import torch
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    b = serving_block(args)
    b.update({"n_gpus": 1, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic"})
    print(json.dumps(b), flush=True)


def run_volume_sweep(args):
    """The clustered-points workload's 10,000 tiles (drawn from the 100M-point
    layer) rendered over layers of N points from the same mixture, for each N:
    tiles/s, index build time and the traversal's visits per tile (the paper's
    claim that display-driven rendering time hardly depends on data volume,
    Sec. 3.3 and Exp. 1)."""
    import torch
    from paper_2005_12489_gb300 import hv
    sizes = [int(v) for v in args.volume_sweep.split(",")]
    w = WORKLOADS[2]
    ref_pts = gen.gmm_points(w["n_objects"], seed=2, k=64)
    reqs = gen.density_tiles(ref_pts, args.tiles, w["zoom"][0], w["zoom"][1], w["r16"], seed=102)
    del ref_pts
    ctx = hv.hv_create(0)
    mode = hv.HV_MODE_RGBA
    tb = hv.hv_tile_bytes(mode)
    n = len(reqs)
    style = hv.make_style(STYLE_T[:3], STYLE_T[4:7])
    d_req = torch.from_numpy(hv.make_requests(reqs).view(np.uint8).copy()).cuda()
    d_out = torch.empty((n, tb), dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rows = []
    for size in sizes:
        pts = gen.gmm_points(size, seed=2, k=64)
        layer = hv.hv_layer_load_points(ctx, pts)
        del pts
        hv.hv_layer_build_index(layer, hv.HV_INDEX_RTREE)
        info = hv.hv_layer_info_get(layer)
        for _ in range(args.warmup):
            flush.fill_(1)
            hv.hv_render_tiles(layer, d_req, n, mode, hv.HV_INDEX_RTREE, style, d_out, d_out.numel(), stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(k & 255)
            evs[k][0].record(stream)
            hv.hv_render_tiles(layer, d_req, n, mode, hv.HV_INDEX_RTREE, style, d_out, d_out.numel(), stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps

        class _L:
            kind, obj_bytes, n_objects = "points", 8, size
        alg = algorithmic_bytes_per_tile(hv, layer, reqs, torch, args.count_sample_tiles, _L)
        rows.append({"points": size, "tiles_per_s": n / (ms / 1000.0), "ms_per_step": ms,
                     "index_build_ms": info.build_ms, "tree_levels": info.tree_levels,
                     "node_visits_per_tile": alg and alg["node_visits_per_tile"],
                     "leaf_visits_per_tile": alg and alg["leaf_visits_per_tile"],
                     "unique_bytes_read_per_tile": alg and alg["read_per_tile"]})
        hv.hv_layer_free(layer)
    hv.hv_destroy(ctx)
    print(json.dumps({"metric": "tiles/s vs data volume (same tiles)", "unit": "tiles/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "data": "synthetic", "dtype": "int64",
                      "config": {"workload": w["workload"].replace("clustered points 100M", "clustered points N"),
                                 "tiles_from": "the 100M-point layer (seed 2)"},
                      "sweep": rows}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == 5:
        run_serving(args)
    elif args.volume_sweep:
        run_volume_sweep(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
