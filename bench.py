"""Benchmark of the shear-4PCF multipole estimator on one GB300 (or N replicas).

One step = one pass of the whole hot path over one synthetic catalogue: cell grid and
radix sort, neighbour gather of the multipoles, contraction into Upsilon_mu / N,
multiple-counting corrections, and the fourth-order aperture measures (real space formed
on the fly).  Workload: a Gaussian-random-field shear mock of 2e6 galaxies on a 10 deg x
10 deg flat patch (power-law P(l) ~ l^-1.2 on a 4096^2 grid, Kaiser-Squires, shape noise
0.26 per component, weights U[0.5, 1.5]), 10 log radial bins 0.5'-40', n_max = 20;
aperture measures on 129 angular bins and 24 log-spaced aperture radii 1'-32'.

Metric: galaxy pairs per second (pairs with separation inside the radial bins, counted by
the kernels) over the whole step; the contraction TFLOP/s and the mixed-vs-FP64 comparison
are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32] [--impl ours|reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
N_SM = 152
FP32_LANES_PER_SM = 128
N_PHI = 129
AP_RADII = np.geomspace(1.0, 32.0, 24)
METRIC = "galaxy pairs/s + Upsilon contraction TFLOP/s; mixed vs FP64 form at stated rel err"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["source"] = "fallback"
    return d


def measured_traffic(kernel):
    """DRAM bytes (read + write) per launch of a kernel from the committed ncu summaries under
    profiles/: a line 'traffic <kernel> <bytes per launch> <source file> <sha256 prefix>'.  The
    figure is used only while the kernel's source file still has that hash (a changed kernel
    needs a new capture); otherwise None."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            f = line.split()
            if len(f) == 5 and f[0] == "traffic" and f[1] == kernel:
                src = os.path.join(ROOT, "paper_2509_07974_gb300", "csrc", f[3])
                if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == f[4]:
                    return float(f[2])
    return None


def gather_flop_per_pair(nmax):
    """Algorithmic FP32 work of one (centre, neighbour) pair in the gather: complex
    accumulations x u^n (4N+3 values) and x^2 u^n (4N+5), real-weighted w u^m (2N+1),
    |x|^2 u^m (2N+3), w^2 u^m (2N+1), the powers u^1..u^{2N+6} and ~40 for the triple terms."""
    N = nmax
    return 8 * (4 * N + 3) + 8 * (4 * N + 5) + 4 * ((2 * N + 1) + (2 * N + 3) + (2 * N + 1)) + 6 * (2 * N + 6) + 40


def contraction_flop(n_centres, nmax, nb):
    """One complex multiply-add per output element per centre: 8 * centres * 9 (2N+1)^2 nb^3."""
    return 8.0 * n_centres * 9 * (2 * nmax + 1) ** 2 * nb ** 3


def reduced_contraction_flop(n_centres, nmax, nb):
    """The complex multiply-adds the tensor-core contraction computes under the exchange of
    Theta2 and Theta3 (Table tab:4PCFSymm): bin pairs Theta2 <= Theta3 only, and for the eight
    components with offset o = +-1 one more n2 per s (the multipoles the map reaches), i.e.
    (2N+1)^2 + 4N+1 multipole pairs instead of (2N+1)^2; the normalisation keeps (2N+1)^2."""
    pairs = nb * (nb + 1) // 2
    n_sq = (2 * nmax + 1) ** 2
    per_centre = 8 * (n_sq + 4 * nmax + 1) * pairs * nb + n_sq * pairs * nb
    return 8.0 * n_centres * per_centre


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, sm_max_default):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": sm_max_default, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, name in enumerate(names):
            if any(r[5 + k].lower() in ("active", "1") for r in rows):
                reasons.append(name)
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else sm_max_default, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def make_workload(seed_offset=0, n=None):
    """The 2e6-galaxy GRF mock, or (n given) a smaller patch at the same density."""
    import synth
    c = dict(synth.GRF2E6)
    if n and n != c["n"]:
        f = (n / c["n"]) ** 0.5
        c["side"] = c["side"] * f
        c["grid"] = max(256, int(2 ** round(np.log2(c["grid"] * f))))
        c["n"] = n
        c["name"] = "GRF %.3g gal, %.0f'x%.0f' (same density), 10 log bins 0.5'-40', n_max=20" % (n, c["side"], c["side"])
    pos, sh, w = synth.grf_catalog(c["n"], c["side"], c["seed"] + seed_offset, grid=c["grid"])
    edges = synth.log_edges(c["lo"], c["hi"], c["nb"])
    return pos, sh, w, edges, c["nmax"], c


def dist_setup(want_gpu):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if want_gpu else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------------------------------
def oracle_sample(pos, sh, w, edges, nmax, n_centres, seed=0):
    """A bounded sample of the workload for the CPU oracle: n_centres random centres (every
    galaxy stays a neighbour).  Returns (mask, seconds, threads)."""
    import oracle
    oracle.build()
    mask = np.zeros(len(w), np.uint8)
    mask[np.random.default_rng(1234 + seed).choice(len(w), n_centres, replace=False)] = 1
    t0 = time.perf_counter()
    oracle.measure(pos, sh, w, edges, nmax, centre_mask=mask)
    return mask, time.perf_counter() - t0, os.cpu_count()


def pairs_of_mask(pos, edges, mask):
    """Pairs of the sampled centres, counted with a k-d tree (for the oracle's rate)."""
    from scipy.spatial import cKDTree
    t = cKDTree(pos)
    cen = pos[mask.astype(bool)]
    tc = cKDTree(cen)
    hi = tc.count_neighbors(t, np.nextafter(edges[-1], 0))
    lo = tc.count_neighbors(t, np.nextafter(edges[0], 0))
    return int(hi - lo)


def run_reference(args):
    """The oracle (plain FP64 CPU program) on a bounded sample of the same workload."""
    world, rank, _ = dist_setup(False)
    if rank != 0:
        return
    if args.workload == "grf2e6":
        pos, sh, w, edges, nmax, c = make_workload(n=args.n_gal)
        n_c = args.oracle_centres
        name = c["name"]
    else:
        # the first catalogue of the batched workload (its own galaxies as neighbours)
        pos, sh, w, offs, _, _, _, edges, nmax, wc = batched_workload(args.workload, args)
        pos, sh, w = pos[offs[0]:offs[1]], sh[offs[0]:offs[1]], w[offs[0]:offs[1]]
        n_c = min(args.oracle_centres, 40 if args.workload == "batch64" else 12)
        name = wc["workload"] + " (oracle on the first catalogue)"
        c = {"nb": len(edges) - 1}
    mask, _, _ = oracle_sample(pos, sh, w, edges, nmax, n_c)  # warm-up build and page-in
    pairs = pairs_of_mask(pos, edges, mask)
    for _ in range(max(0, args.warmup - 1)):
        oracle_sample(pos, sh, w, edges, nmax, n_c, seed=1)
    times = []
    for k in range(args.steps):
        _, dt, cores = oracle_sample(pos, sh, w, edges, nmax, n_c, seed=0)
        times.append(dt)
    t = sum(times) / len(times)
    value = pairs / t
    sample = "%d random centres of the %d-galaxy catalogue (all galaxies as neighbours), %d pairs" % (
        n_c, len(w), pairs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "n_gal": len(w), "n_bins": c["nb"], "n_max": nmax,
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def third_order(dev, stream, flush, args):
    """The shear 3PCF (order 3 of App. F, ext4pcf_measure3) on a 2e5-galaxy GRF at the density
    of the main workload (190' x 190'), its 10 log bins 0.5'-40' and n_max = 20, every galaxy a
    centre: FP32 gather, FP64 contraction.  W warm-up calls, max(K, 3) timed calls with L2
    flushed between them; pairs per call from one ext4pcf_measure call with statistics on the
    same catalogue and bins (the same neighbour pairs), outside the timed region."""
    import torch

    import synth
    from paper_2509_07974_gb300 import ext4pcf
    c = synth.GRF2E6
    n = 200_000
    side = c["side"] * (n / c["n"]) ** 0.5
    pos, sh, w = synth.grf_catalog(n, side, c["seed"] + 3, grid=1024)
    edges = np.ascontiguousarray(synth.log_edges(c["lo"], c["hi"], c["nb"]))
    nb, nmax = c["nb"], c["nmax"]
    tp, ts, tw = (torch.tensor(a, device=dev) for a in (pos, sh, w))
    est = ext4pcf.Estimator(0, "f16x3", stream=stream)
    ups3 = torch.zeros((5, 2 * nmax + 1, nb, nb, 2), dtype=torch.float64, device=dev)
    st = ext4pcf.Stats()
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(nb, nmax), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        ext4pcf.ext4pcf_measure(est.ctx, tp, ts, tw, n, edges, nb, nmax, None, 1, None, ups, None, st)
    pairs = float(st.as_dict()["pairs"])
    del ups

    def call(p, s_, w_, out):
        ext4pcf.ext4pcf_measure3(est.ctx, p, s_, w_, n, edges, nb, nmax, out)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            ups3.zero_()
            call(tp, ts, tw, ups3)
        torch.cuda.synchronize()
        n_t = max(args.steps, 3)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_t)]
        for k in range(n_t):
            flush.fill_(float(k))
            ups3.zero_()
            evs[k][0].record(stream)
            call(tp, ts, tw, ups3)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / n_t
    # end to end through the user's calls: the catalogue from pinned host memory to the device,
    # the measurement, the multipoles back to the host
    hp, hs, hw = (torch.tensor(a).pin_memory() for a in (pos, sh, w))
    host = torch.zeros(ups3.shape, dtype=torch.float64).pin_memory()
    e2e_t = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            dp, ds, dw = (x.to(dev, non_blocking=True) for x in (hp, hs, hw))
            ups3.zero_()
            call(dp, ds, dw, ups3)
            host.copy_(ups3, non_blocking=True)
        stream.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e = sum(e2e_t) / len(e2e_t)
    est.close()
    return {"workload": "shear 3PCF: GRF 2e5 gal, %.0f'x%.0f' (the main density), 10 log bins 0.5'-40', n_max=20, "
                        "every galaxy a centre" % (side, side),
            "pairs_per_call": pairs, "value": pairs / (ms / 1e3), "unit": "pairs/s", "ms_per_call": ms,
            "dtype": "f32 gather, f64 contraction", "l2": "flushed between calls (256 MB write)",
            "e2e": {"value": pairs / e2e, "unit": "pairs/s", "h2d_bytes_per_step": int(3 * n * 8 + n * 8),
                    "d2h_bytes_per_step": int(host.numel() * 8)},
            "cpu_baseline": None}


def direct_estimator(est, tp, ts, tw, pos, sh, w, side, dev, stream, flush, args, baselines):
    """Direct <M_ap^4> estimator (Sect. 5.2, Eq. MapDirectEstimator) on the same catalogue:
    24 log radii 1'-32', aperture lattices of spacing theta at least 4 theta inside the field,
    one ext4pcf_map_direct call per pass (grid build included).  Timed on its own, after the
    main measurement: W warm-up passes, max(K, 5) timed passes with L2 flushed between them."""
    import torch

    import synth
    from paper_2509_07974_gb300 import ext4pcf
    cfg = synth.DIRECT
    radii = np.ascontiguousarray(synth.direct_radii())
    lat = [ext4pcf.aperture_lattice((0.0, 0.0, side, side), t, cfg["spacing"] * t) for t in radii]
    offs = np.zeros(len(radii) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(x) for x in lat])
    cen_h = np.ascontiguousarray(np.vstack(lat))
    cen = torch.tensor(cen_h, device=dev)
    mom = torch.zeros((len(radii), 8), dtype=torch.float64, device=dev)
    rec = torch.zeros((int(offs[-1]), 8), dtype=torch.float64, device=dev)

    def call(p, s_, w_, c_, m_):
        ext4pcf.ext4pcf_map_direct(est.ctx, p, s_, w_, len(w), radii, len(radii), c_, offs, rec, m_)

    mom.zero_()
    call(tp, ts, tw, cen, mom)
    torch.cuda.synchronize()
    pairs = float(rec[:, 6].sum().item())
    for _ in range(args.warmup):
        mom.zero_()
        call(tp, ts, tw, cen, mom)
    torch.cuda.synchronize()
    n_t = max(args.steps, 5)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_t)]
    for k in range(n_t):
        flush.fill_(float(k))
        mom.zero_()
        evs[k][0].record(stream)
        call(tp, ts, tw, cen, mom)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / n_t
    # end to end: catalogue and centres from pinned host memory, moments read back
    hp, hs, hw = (torch.tensor(a).pin_memory() for a in (pos, sh, w))
    hc = torch.tensor(cen_h).pin_memory()
    hm = np.zeros((len(radii), 8))
    e2e_t = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hm[:] = 0.0
        call(hp, hs, hw, hc, hm)
        e2e_t.append(time.perf_counter() - t0)
    e2e = sum(e2e_t) / len(e2e_t)
    m = mom.cpu().numpy()
    out = {"workload": cfg["name"], "radii": len(radii), "apertures": int(offs[-1]),
           "pairs_per_pass": pairs, "value": pairs / (ms / 1e3), "unit": "aperture-galaxy pairs/s",
           "ms_per_pass": ms, "dtype": "f32 terms, compensated f32 power sums, f64 per aperture",
           "l2": "flushed between passes (256 MB write)",
           "e2e": {"value": pairs / e2e, "unit": "aperture-galaxy pairs/s",
                   "h2d_bytes_per_step": int(hp.numel() * 8 + hs.numel() * 8 + hw.numel() * 8 + hc.numel() * 8),
                   "d2h_bytes_per_step": int(hm.nbytes)},
           "map4_by_radius": {"%.2f" % radii[i]: float(m[i, 5]) for i in (0, 12, 23)},
           "cpu_baseline": None}
    if baselines:
        import oracle
        t8 = float(radii[16])
        pick = np.random.default_rng(5).choice(len(lat[16]), size=6, replace=False)
        t0 = time.perf_counter()
        opairs = sum(oracle.aperture_record(pos, sh, w, lat[16][i], t8)[6] for i in pick)
        odt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": opairs / odt, "unit": "aperture-galaxy pairs/s", "cores": 1,
                               "kind": "oracle",
                               "sample": "6 apertures of radius %.2f' (numpy, all galaxies tested), %d pairs, %.1f s"
                                         % (t8, opairs, odt)}
    return out


# ------------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_2509_07974_gb300 import build, ext4pcf

    world, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    pk = peaks()
    pos, sh, w, edges, nmax, c = make_workload(seed_offset=rank, n=args.n_gal)
    nb = len(edges) - 1
    tp = torch.tensor(pos, device=dev)
    ts = torch.tensor(sh, device=dev)
    tw = torch.tensor(w, device=dev)
    stream = torch.cuda.current_stream(dev)
    est = ext4pcf.Estimator(local, args.precision, stream=stream)
    ups = torch.zeros(ext4pcf.Estimator.ups_shape(nb, nmax), dtype=torch.float64, device=dev)
    xia = torch.zeros((1, nb, 3, 2), dtype=torch.float64, device=dev)
    edges_c = np.ascontiguousarray(edges)
    ap = np.ascontiguousarray(AP_RADII)
    m4 = np.zeros((len(ap), 8, 2))
    eb = np.zeros((len(ap), 16))
    disc = np.zeros((len(ap), 16))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    # profiling aid: a seeded subset of the galaxies act as centres (all stay neighbours)
    cmask = None
    if args.centres is not None:
        sel = np.random.default_rng(7).choice(len(w), size=min(args.centres, len(w)), replace=False)
        hm = np.zeros(len(w), dtype=np.uint8)
        hm[sel] = 1
        cmask = torch.tensor(hm, device=dev)

    def step(stats=None):
        ups.zero_()
        xia.zero_()
        ext4pcf.ext4pcf_measure(est.ctx, tp, ts, tw, len(w), edges_c, nb, nmax, None, 1, cmask, ups, xia, stats)
        ext4pcf.ext4pcf_to_map4(est.ctx, ups, edges_c, nb, nmax, N_PHI, ap, len(ap), xia, m4, eb, disc)

    # pair count of the workload (one untimed call with statistics)
    st = ext4pcf.Stats()
    step(st)
    torch.cuda.synchronize()
    pairs = st.as_dict()["pairs"]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps (outside the per-step events).  Each
    # step also collects the library's per-phase device times (events recorded on the
    # library's stream around every wave's gather, contraction and corrections; no host
    # synchronisation until the end of the call)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sts = [ext4pcf.Stats() for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as cs:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            step(sts[k])
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier(world)
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    sd = [x.as_dict() for x in sts]
    bd = {k: sum(d[k] for d in sd) / len(sd) for k in sd[0]}  # per-step averages
    log("rank %d: per-step phases %s" % (rank, bd))
    dev_ms_max = max_over_ranks(dev_ms, world, dev)
    pairs_all = sum_over_ranks(float(pairs) * args.steps, world, dev)
    value = pairs_all / (dev_ms_max / 1e3)
    clocks = cs.summary(pk.get("sm_max_mhz", 2070.0))

    # end to end through the C ABI: inputs from pinned host buffers (copied inside the call),
    # results of the step (aperture measures) read back to the host
    hp = torch.tensor(pos).pin_memory()
    hs = torch.tensor(sh).pin_memory()
    hw = torch.tensor(w).pin_memory()
    hmask = cmask.cpu().pin_memory() if cmask is not None else None
    e2e_t = []
    for k in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ups.zero_()
        xia.zero_()
        ext4pcf.ext4pcf_measure(est.ctx, hp, hs, hw, len(w), edges_c, nb, nmax, None, 1, hmask, ups, xia, None)
        ext4pcf.ext4pcf_to_map4(est.ctx, ups, edges_c, nb, nmax, N_PHI, ap, len(ap), xia, m4, eb, disc)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e = sum(e2e_t) / len(e2e_t)
    h2d = hp.numel() * 8 + hs.numel() * 8 + hw.numel() * 8 + (hmask.numel() if hmask is not None else 0)
    d2h = m4.nbytes + eb.nbytes + disc.nbytes

    direct = third = None
    if rank == 0:
        direct = direct_estimator(est, tp, ts, tw, pos, sh, w, c["side"], dev, stream, flush, args,
                                  world == 1 and not args.no_baselines)
        third = third_order(dev, stream, flush, args)

    # rooflines of the two dominant kernels, algorithmic FLOP per launch over the average
    # launch duration in the timed steps.  Gather: FP32 work on the CUDA cores against the
    # FP32 FMA pipe.  Contraction: complex multiply-adds of the outputs on the tensor cores
    # against the TF32 rate (measured sustained bf16 x the nominal tf32/bf16 ratio 1.1/2.25;
    # the 3xTF32 form issues three MMAs per algorithmic product).
    waves = max(1, bd["waves"])
    flop_pair = gather_flop_per_pair(nmax)
    g_ms = bd["ms_gather"] / waves
    g_ach = flop_pair * pairs / waves / (g_ms / 1e3) / 1e12
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    tc_form = args.precision in ("tf32", "3xtf32", "bf16x3", "f16x3")
    c_flop_full = contraction_flop(bd["centres"], nmax, nb)
    c_flop = reduced_contraction_flop(bd["centres"], nmax, nb) if tc_form else c_flop_full
    c_ms = bd["ms_contract"] / waves
    contraction_tflops = c_flop / (bd["ms_contract"] / 1e3) / 1e12 if bd["ms_contract"] > 0 else None
    passes = {"3xtf32": 3, "bf16x3": 3, "f16x3": 3, "tf32": 1}.get(args.precision, 1)
    # the tensor rate of the contraction's operand type: kind::f16 (fp16 / bf16 halves) runs at
    # the measured bf16 rate, kind::tf32 at that rate times the nominal ratio 1.1/2.25
    f16_kind = args.precision in ("f16x3", "bf16x3")
    tf32_peak = pk.get("bf16_tflops_sustained", 1700.0) * (1.0 if f16_kind else 1.1 / 2.25)
    roof_g = {"bound": "alu", "kernel": "gather", "achieved": g_ach, "peak": fp32_peak, "unit": "TFLOP/s",
              "frac": g_ach / fp32_peak, "traffic": None, "ms_per_launch": g_ms,
              "peak_note": "FP32 FMA pipe: 152 SMs x 128 lanes x 2 FLOP x max SM clock (%s MHz)"
                           % pk.get("sm_max_mhz", 2070.0),
              "algorithmic_flop_per_pair": flop_pair}
    roof_c = {"bound": "tensor", "kernel": "contraction", "achieved": contraction_tflops, "peak": tf32_peak,
              "unit": "TFLOP/s", "frac": (contraction_tflops or 0.0) / tf32_peak, "traffic": None,
              "ms_per_launch": c_ms,
              "frac_issued": (contraction_tflops or 0.0) * passes / tf32_peak,
              "passes": passes,
              "peak_note": ("kind::f16 dense: measured sustained bf16 (%s TFLOP/s, %s)"
                            % (pk.get("bf16_tflops_sustained"), pk.get("source"))) if f16_kind else
                           ("tf32 dense: measured sustained bf16 (%s TFLOP/s, %s) x the nominal ratio 1.1/2.25 "
                            "(not a measured tf32 rate)" % (pk.get("bf16_tflops_sustained"), pk.get("source"))),
              "algorithmic_flop_per_centre": c_flop / max(1, bd["centres"]),
              "algorithmic_note": ("complex multiply-adds of the symmetry-reduced contraction (bin pairs "
                                   "Theta2 <= Theta3); all ordered triples would be %.4g FLOP per centre, "
                                   "%.3g TFLOP/s equivalent" % (c_flop_full / max(1, bd["centres"]),
                                   c_flop_full / (bd["ms_contract"] / 1e3) / 1e12 if bd["ms_contract"] > 0 else 0.0))
                                  if tc_form else "complex multiply-adds of all ordered bin triples"}
    # DRAM bytes (read + write) of one full-size launch of the default configuration, from the
    # committed ncu summaries (null when the kernel source changed since the capture)
    if args.n_gal is None and args.centres is None:
        roof_g["traffic"] = measured_traffic("gather_kernel")
        roof_c["traffic"] = measured_traffic("contract_h16_kernel" if args.precision == "f16x3"
                                             else "contract_tc_kernel" if tc_form else "contract_kernel")
        roof_g["traffic_unit"] = roof_c["traffic_unit"] = "bytes per launch (DRAM read + write, ncu)"
    roof_main, roof_other = (roof_c, roof_g) if c_ms >= g_ms else (roof_g, roof_c)

    fp64_info = None
    cpu = None
    if rank == 0 and world == 1 and not args.no_baselines:
        # FP64 GPU form on a sample of centres, for the mixed-vs-FP64 comparison
        mask = np.zeros(len(w), np.uint8)
        mask[np.random.default_rng(77).choice(len(w), args.fp64_centres, replace=False)] = 1
        tm = torch.tensor(mask, device=dev)
        e64 = ext4pcf.Estimator(local, "fp64", stream=stream)
        u64 = torch.zeros_like(ups)
        s64 = ext4pcf.Stats()
        ext4pcf.ext4pcf_measure(e64.ctx, tp, ts, tw, len(w), edges_c, nb, nmax, None, 1, tm, u64, None, s64)
        torch.cuda.synchronize()
        s64 = s64.as_dict()
        umx = torch.zeros_like(ups)
        smx = ext4pcf.Stats()
        ext4pcf.ext4pcf_measure(est.ctx, tp, ts, tw, len(w), edges_c, nb, nmax, None, 1, tm, umx, None, smx)
        torch.cuda.synchronize()
        smx = smx.as_dict()
        a = torch.view_as_complex(umx).cpu().numpy()
        b = torch.view_as_complex(u64).cpu().numpy()[0]
        a = a[0]
        floor = np.sqrt(np.mean(np.abs(b) ** 2, axis=(1, 2), keepdims=True))
        scale = np.abs(b).reshape(9, -1).max(axis=1).reshape(9, 1, 1, 1, 1, 1)
        den = np.maximum(np.maximum(np.abs(b), floor), 1e-12 * scale)
        err = float((np.abs(a - b) / np.where(den > 0, den, 1)).max())
        fp64_info = {"centres": args.fp64_centres, "pairs": s64["pairs"],
                     "fp64_pairs_per_s": s64["pairs"] / (s64["ms_total"] / 1e3),
                     "mixed_pairs_per_s_same_sample": smx["pairs"] / (smx["ms_total"] / 1e3),
                     "speedup_mixed_vs_fp64": (s64["ms_total"] / smx["ms_total"]),
                     "max_rel_err_mixed_vs_fp64": err}
        e64.close()
        # CPU oracle on a bounded sample
        omask, odt, cores = oracle_sample(pos, sh, w, edges, nmax, args.oracle_centres)
        opairs = pairs_of_mask(pos, edges, omask)
        cpu = {"value": opairs / odt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": "%d random centres of the %d-galaxy catalogue (all galaxies as neighbours), %d pairs, %.1f s"
                         % (args.oracle_centres, len(w), opairs, odt)}

    # kernels per step: those of ext4pcf_measure (counted by the library) plus those of
    # ext4pcf_to_map4: angle table + (norm, gamma, integrate) per chunk of radial triples + finish
    nph2 = N_PHI * N_PHI
    chunk = min(nb ** 3, max(1, (256 << 20) // (nph2 * 8 * 16)))
    map4_launches = 2 + 3 * ((nb ** 3 + chunk - 1) // chunk)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
                "data": "synthetic",
                "config": {"workload": c["name"], "n_gal": len(w), "n_bins": nb, "n_max": nmax,
                           "precision": args.precision, "n_phi": N_PHI, "apertures": len(ap),
                           "pairs_per_step": pairs, "l2": "flushed between steps (256 MB write)",
                           **({"centres": args.centres} if args.centres is not None else {}),
                           "parallelism": "one catalogue per GPU" if world > 1 else "1 GPU"},
                "contraction_tflops": contraction_tflops,
                "pairs_per_s_gather": pairs / (bd["ms_gather"] / 1e3) if bd["ms_gather"] > 0 else None,
                "breakdown_ms": {k: bd[k] for k in ("ms_grid", "ms_gather", "ms_contract", "ms_correct", "ms_total")},
                "wall_s": t_wall,
                "e2e": {"value": pairs / e2e, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "roofline": roof_main,
                "roofline_secondary": roof_other,
                "fp64_form": fp64_info,
                "cpu_baseline": cpu,
                "next_rows": {"map_direct": direct, "third_order": third},
                "clocks": clocks,
                "gpu_launches": int((bd["launches"] + map4_launches) * args.steps)}
        print(json.dumps(line), flush=True)
    est.close()


# ------------------------------------------------------------------------------------------
# Batched and survey workloads (ext4pcf_measure_batch, one captured CUDA graph per step)
def batched_workload(kind, args, seed_offset=0):
    """(pos, shear, w, cat_offsets, out_slot or None, n_out, centre mask, edges, n_max, config)
    of the batched form (64 uneven GRF mocks, one slot each) or the survey (1e8 lognormal
    galaxies in 10 x 10 patches with 120' margins, all patches in one slot).  The centres are
    a seeded sample: per mock (or per patch core) `per_cat` of its galaxies."""
    import synth
    rng = np.random.default_rng(4321 + seed_offset)
    if kind == "batch64":
        c = synth.BATCH64
        pos, sh, w, offs, edges, nmax = synth.batch64_workload(n_mocks=args.n_cat)
        per_cat = args.centres_per_cat or 1024
        mask = np.zeros(len(w), np.uint8)
        for k in range(len(offs) - 1):
            nk = int(offs[k + 1] - offs[k])
            mask[offs[k] + rng.choice(nk, min(per_cat, nk), replace=False)] = 1
        slots, n_out = None, len(offs) - 1
        cfg = {"workload": c["name"], "n_cat": len(offs) - 1, "n_gal": len(w),
               "galaxies_per_mock": [int(v) for v in (np.min(np.diff(offs)), np.max(np.diff(offs)))],
               "centres_per_mock": per_cat}
    else:
        c = synth.SURVEY
        n = args.n_gal or c["n"]
        side = c["side"] * (n / c["n"]) ** 0.5
        pos, sh, w, offs, core, edges, nmax = synth.survey_workload(n=n, side=side)
        n_side = int(round((len(offs) - 1) ** 0.5))
        per_cat = args.centres_per_cat or 128
        mask = np.zeros(len(w), np.uint8)
        for k in range(len(offs) - 1):
            cidx = offs[k] + np.flatnonzero(core[offs[k]:offs[k + 1]])
            mask[rng.choice(cidx, min(per_cat, len(cidx)), replace=False)] = 1
        slots, n_out = np.zeros(len(offs) - 1, np.int32), 1
        cfg = {"workload": c["name"] if n == c["n"] else "lognormal survey %.3g gal (same density), %.0f'x%.0f', "
               "%dx%d patches + 120' margins, 12 log bins 0.5'-120', n_max=30" % (n, side, side, n_side, n_side),
               "n_gal": int(n), "n_gal_patched": len(w), "n_cat": len(offs) - 1, "centres_per_patch": per_cat}
    return pos, sh, w, offs, slots, n_out, mask, edges, nmax, cfg


def run_batched(args, kind):
    import torch

    from paper_2509_07974_gb300 import build, ext4pcf

    world, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    pk = peaks()
    t_gen = time.perf_counter()
    pos, sh, w, offs, slots, n_out, mask, edges, nmax, wcfg = batched_workload(kind, args, seed_offset=rank)
    log("rank %d: workload generated in %.1f s (%d galaxies, %d catalogues)" % (rank, time.perf_counter() - t_gen,
                                                                                len(w), len(offs) - 1))
    nb = len(edges) - 1
    n_cat = len(offs) - 1
    tp = torch.tensor(pos, device=dev)
    ts = torch.tensor(sh, device=dev)
    tw = torch.tensor(w, device=dev)
    hmask = torch.tensor(mask).pin_memory()  # pinned host mask: counts known on the host, copy in the graph
    stream = torch.cuda.Stream(dev)
    cfg = ext4pcf.Config(device=local, stream=stream.cuda_stream, precision=ext4pcf.PRECISION[args.precision],
                         autotune=1, workspace_bytes=0, timeout_cycles=0, deterministic=1, wave_centres=0)
    ctx = ext4pcf.ext4pcf_create(cfg)
    shape = (n_out,) + tuple(ext4pcf.Estimator.ups_shape(nb, nmax)[1:])
    ups = torch.zeros(shape, dtype=torch.float64, device=dev)
    xia = torch.zeros((n_out, nb, 3, 2), dtype=torch.float64, device=dev)
    edges_c = np.ascontiguousarray(edges)
    offs_c = np.ascontiguousarray(offs, dtype=np.int64)
    slots_c = None if slots is None else np.ascontiguousarray(slots, dtype=np.int32)
    n_out_arg = n_out if slots is not None else 0
    want_map4 = kind == "survey"
    ap = np.ascontiguousarray(AP_RADII)
    m4 = np.zeros((len(ap), 8, 2))
    eb = np.zeros((len(ap), 16))
    disc = np.zeros((len(ap), 16))

    def measure(stats=None, p=tp, s=ts, ww=tw):
        ext4pcf.ext4pcf_measure_batch(ctx, p, s, ww, len(w), edges_c, nb, nmax, offs_c, n_cat, slots_c, n_out_arg,
                                      hmask, ups, xia, stats)

    # the first call autotunes the wave size (timed trial waves) and sizes every buffer; the
    # second gives the steady-state phase breakdown and the pair count
    with torch.cuda.stream(stream):
        st0 = ext4pcf.Stats()
        measure(st0)
        st = ext4pcf.Stats()
        ups.zero_()
        xia.zero_()
        measure(st)
    stream.synchronize()
    bd = st.as_dict()
    pairs = bd["pairs"]
    log("rank %d: %s" % (rank, bd))
    # one step = the captured graph (zero the outputs, the batched measure) [+ the FP64
    # aperture measures of the survey's Upsilon, which read results back to the host]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
        ups.zero_()
        xia.zero_()
        measure()
    if ext4pcf.ext4pcf_synchronize(ctx) != ext4pcf.EXT4PCF_OK:
        raise RuntimeError("status after capture")

    def step():
        with torch.cuda.stream(stream):  # the graph replays on the current stream
            g.replay()
            if want_map4:
                ext4pcf.ext4pcf_to_map4(ctx, ups[0], edges_c, nb, nmax, N_PHI, ap, len(ap), xia[0], m4, eb, disc)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as cs:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    barrier(world)
    if ext4pcf.ext4pcf_synchronize(ctx) != ext4pcf.EXT4PCF_OK:
        raise RuntimeError("status after the timed steps")
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    dev_ms_max = max_over_ranks(dev_ms, world, dev)
    pairs_all = sum_over_ranks(float(pairs) * args.steps, world, dev)
    value = pairs_all / (dev_ms_max / 1e3)
    clocks = cs.summary(pk.get("sm_max_mhz", 2070.0))

    # end to end through the C ABI: inputs from pinned host buffers (copied inside the call),
    # the xi accumulators (and the survey's aperture measures) read back to the host
    hp = torch.tensor(pos).pin_memory()
    hs = torch.tensor(sh).pin_memory()
    hw = torch.tensor(w).pin_memory()
    hxi = np.zeros((n_out, nb, 3, 2))
    e2e_t = []
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            ups.zero_()
            hxi[:] = 0
            ext4pcf.ext4pcf_measure_batch(ctx, hp, hs, hw, len(w), edges_c, nb, nmax, offs_c, n_cat, slots_c,
                                          n_out_arg, hmask, ups, hxi, None)
            if want_map4:
                ext4pcf.ext4pcf_to_map4(ctx, ups[0], edges_c, nb, nmax, N_PHI, ap, len(ap),
                                        np.ascontiguousarray(hxi[0]), m4, eb, disc)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e = sum(e2e_t) / len(e2e_t)
    h2d = hp.numel() * 8 + hs.numel() * 8 + hw.numel() * 8 + hmask.numel()
    d2h = hxi.nbytes + ((m4.nbytes + eb.nbytes + disc.nbytes) if want_map4 else 0)

    # rooflines of the two dominant kernels from the steady-state call's phase times
    waves = max(1, bd["waves"])
    flop_pair = gather_flop_per_pair(nmax)
    g_ms = bd["ms_gather"] / waves
    g_ach = flop_pair * pairs / (bd["ms_gather"] / 1e3) / 1e12
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    c_flop = reduced_contraction_flop(bd["centres"], nmax, nb)
    c_tflops = c_flop / (bd["ms_contract"] / 1e3) / 1e12 if bd["ms_contract"] > 0 else None
    peak_c = pk.get("bf16_tflops_sustained", 1700.0)
    roof_g = {"bound": "alu", "kernel": "gather", "achieved": g_ach, "peak": fp32_peak, "unit": "TFLOP/s",
              "frac": g_ach / fp32_peak, "traffic": None, "ms_per_launch": g_ms,
              "peak_note": "FP32 FMA pipe: 152 SMs x 128 lanes x 2 FLOP x max SM clock",
              "algorithmic_flop_per_pair": flop_pair}
    roof_c = {"bound": "tensor", "kernel": "contraction", "achieved": c_tflops, "peak": peak_c, "unit": "TFLOP/s",
              "frac": (c_tflops or 0.0) / peak_c, "frac_issued": 3 * (c_tflops or 0.0) / peak_c, "passes": 3,
              "traffic": None, "ms_per_launch": bd["ms_contract"] / waves,
              "peak_note": "kind::f16 dense: measured sustained bf16 (%s TFLOP/s, %s)"
                           % (pk.get("bf16_tflops_sustained"), pk.get("source")),
              "algorithmic_flop_per_centre": c_flop / max(1, bd["centres"])}
    roof_main, roof_other = (roof_c, roof_g) if bd["ms_contract"] >= bd["ms_gather"] else (roof_g, roof_c)

    tree_info = None
    if kind == "survey" and rank == 0:
        # the tree approximation (Sect. 3.2, App. F.3) with the paper's setting for its survey
        # (resolutions 0.5', 1', 2', r_min = 40) on the same centres, against the exact result
        exact = torch.view_as_complex(ups[0]).cpu().numpy()
        tcfg = ext4pcf.Config(device=local, stream=stream.cuda_stream, precision=ext4pcf.PRECISION[args.precision],
                              autotune=0, workspace_bytes=0, timeout_cycles=0, deterministic=1,
                              wave_centres=int(bd["wave_centres"]), tree_delta1=0.5, tree_levels=3, tree_rmin=40.0)
        tctx = ext4pcf.ext4pcf_create(tcfg)
        tst = ext4pcf.Stats()
        t_ms = []
        for k in range(2):
            with torch.cuda.stream(stream):
                ups.zero_()
                xia.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ext4pcf.ext4pcf_measure_batch(tctx, tp, ts, tw, len(w), edges_c, nb, nmax, offs_c, n_cat, slots_c,
                                              n_out_arg, hmask, ups, xia, tst if k else None)
                e1.record(stream)
            stream.synchronize()
            t_ms.append(e0.elapsed_time(e1))
        ext4pcf.ext4pcf_destroy(tctx)
        approx = torch.view_as_complex(ups[0]).cpu().numpy()
        floor = np.sqrt(np.mean(np.abs(exact) ** 2, axis=(1, 2), keepdims=True))
        den = np.maximum(np.abs(exact), floor)
        err = np.abs(approx - exact) / np.where(den > 0, den, 1.0)
        tsd = tst.as_dict()
        tree_info = {"setting": "Delta_d = 0.5', 1', 2'; r_min = 40 (the paper's DES setting)",
                     "ms_measure": t_ms[-1], "ms_measure_exact": bd["ms_total"],
                     "speedup_vs_exact": bd["ms_total"] / t_ms[-1],
                     "pairs_exact": pairs, "pairs_tree": tsd["pairs"],
                     "rel_err_vs_exact_max": float(err.max()), "rel_err_vs_exact_median": float(np.median(err)),
                     "metric": "|tree - exact| / max(|exact|, rms over (n2, n3)) over every Upsilon entry",
                     "breakdown_ms": {k: tsd[k] for k in ("ms_grid", "ms_gather", "ms_contract", "ms_correct")}}
        del exact, approx, err, den

    cpu = None
    if rank == 0 and world == 1 and not args.no_baselines:
        # the oracle on a bounded sample: centres of the first catalogue (its galaxies only)
        a, b = int(offs[0]), int(offs[1])
        n_c = min(args.oracle_centres, 40 if kind == "batch64" else 12)
        omask, odt, cores = oracle_sample(pos[a:b], sh[a:b], w[a:b], edges, nmax, n_c)
        opairs = pairs_of_mask(pos[a:b], edges, omask)
        cpu = {"value": opairs / odt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
               "sample": "%d random centres of the first catalogue (%d galaxies, all neighbours), %d pairs, %.1f s"
                         % (n_c, b - a, opairs, odt)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(wcfg, **{"n_bins": nb, "n_max": nmax, "precision": args.precision,
                                        "centres": int(bd["centres"]), "pairs_per_step": pairs,
                                        "waves": int(bd["waves"]), "wave_centres": int(bd["wave_centres"]),
                                        "wave_size": "autotuned over 2048, 4096, 8192, 16384 centres",
                                        "graph": "one captured CUDA graph per step (grids, packed waves, "
                                                 "expansion, corrections)",
                                        "l2": "flushed between steps (256 MB write)",
                                        "parallelism": "one workload per GPU" if world > 1 else "1 GPU"}),
                "contraction_tflops": c_tflops,
                "breakdown_ms": {k: bd[k] for k in ("ms_grid", "ms_gather", "ms_contract", "ms_correct", "ms_total")},
                "wall_s": t_wall,
                "e2e": {"value": pairs / e2e, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "roofline": roof_main, "roofline_secondary": roof_other, "cpu_baseline": cpu,
                "clocks": clocks,
                "gpu_launches": int(bd["launches"] * args.steps)}
        if want_map4:
            line["map4_by_radius"] = {"%.2f" % ap[i]: float(m4[i, 0, 0]) for i in (0, len(ap) // 2, len(ap) - 1)}
        if tree_info is not None:
            line["tree"] = tree_info
        print(json.dumps(line), flush=True)
    ext4pcf.ext4pcf_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16x3", choices=["fp64", "fp32", "tf32", "3xtf32", "bf16x3", "f16x3"])
    ap.add_argument("--oracle-centres", type=int, default=2000)
    ap.add_argument("--fp64-centres", type=int, default=4096)
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--centres", type=int, default=None,
                    help="profiling aid: only this many (seeded random) galaxies act as centres")
    ap.add_argument("--workload", default="grf2e6", choices=["grf2e6", "batch64", "survey"],
                    help="grf2e6: the 2e6-galaxy GRF mock (default); batch64: 64 uneven GRF mocks in one batched "
                         "call; survey: 1e8 lognormal galaxies in 10x10 patches with 120' margins")
    ap.add_argument("--centres-per-cat", type=int, default=None,
                    help="batch64 / survey: sampled centres per mock (1024) or per patch core (128)")
    ap.add_argument("--n-cat", type=int, default=64, help="batch64: number of mocks")
    ap.add_argument("--n-gal", type=int, default=None,
                    help="smaller catalogue at the same density (profiling); default 2e6")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "grf2e6":
        run_batched(args, args.workload)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
