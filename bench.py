#!/usr/bin/env python
"""Throughput of the GB300 Haar-tSVD path: denoised megapixels per second.

Workload (one step, default): three 3840x2160 RGB uint8 images (seeded synthetic, Poisson-Gaussian
noise a=0.01 at b = 10^2, 25^2, 50^2, sigma = sqrt(b) given), each denoised by one C-ABI call:
grouping (ps 8, stride 3, window 31, K 32), global t-SVD bases, Haar + t-SVD projection, hard
threshold, inverse and aggregation. --workload picks the other workloads (512x512 with sigma
estimated, batches, VJP, video, sweeps).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]

With --gpus N > 1 launch under torchrun: each rank denoises its own copy of the workload
(replicas, weak scaling); the reported value is the whole job's megapixels over the slowest
rank's device time. --impl reference times the FP64 CPU oracle on all host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "denoised megapixels/sec at oracle-matched PSNR (±0.01 dB); batched & VJP vs plain"
UNIT = "MP/s"
CONFIGS = {
    "rgb512": {"workload": "rgb512_pg_sigma_est", "image": "512x512x3 uint8", "noise": "poisson-gaussian a=0.01 b=15^2",
               "sigma": "estimated (patch-covariance eigenvalues)", "ps": 8, "stride": 2, "window": 31, "K": 32,
               "groups_per_image": 64009},
    "rgb4k": {"workload": "rgb3840x2160_pg_3levels", "image": "3 x 3840x2160x3 uint8 per step",
              "noise": "poisson-gaussian a=0.01, b in {10^2, 25^2, 50^2}", "sigma": "given (sqrt(b))",
              "ps": 8, "stride": 3, "window": 31, "K": 32, "groups_per_image": 919601},
}


def workload_config(name: str) -> dict:
    return dict(CONFIGS[name])


FLUSH_BYTES = 256 << 20          # > 129 MB L2, written between timed steps (untimed)
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (Blackwell)
MAX_SM_MHZ = 2070.0              # GB300 maximum SM clock


# DRAM bytes (read + write) of one launch of the forward filter kernel, from one ncu capture of
# the current kernel (dram__bytes_read.sum + dram__bytes_write.sum) on the 1920x1080x3 workload,
# which has the 3840x2160 frames' geometry and tile edge; a 3840x2160 launch scales it by its
# groups (919,601 / 229,401: the traffic is the tile partials and indices, both proportional).
FILTER_DRAM_BYTES = {"rgb1080": 37.154816e6 + 304.592384e6,
                     "rgb4k": (37.154816e6 + 304.592384e6) * 919601 / 229401}


def volume_flops_per_group(K: int) -> int:
    """Algorithmic FP32 flops of one group of 4 x 4 x 4 cubes: per cube and direction the per-slice
    projections (slices 0 and 2 real, 2 x 64 MACs each; slice 1 complex, 2 x 64 complex MACs: 1,536
    flop) and the tube DFTs (384 flop), the Haar butterflies (4 flop, K - 1 per fibre and direction,
    64 fibres) and one compare per coefficient. K = 32: 140,800."""
    return K * 2 * (1536 + 384) + 2 * 4 * (K - 1) * 64 + K * 64


def measured_peak(key: str):
    """A peak from the measured MEASURED_PEAKS.json beside this file, or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return None


def filter_flops_per_group(C: int, K: int) -> int:
    """Algorithmic FP32 flops of one group in the structured per-Fourier-slice form:
    t-SVD projections (per patch and direction: 10,240 for C=3, 2,048 for C=1), channel DFTs
    (C=3: 17 flop per pixel and direction), Haar butterflies (4 flop, K-1 per fibre and direction)
    and one compare per coefficient. C=3, K=32: 778,752."""
    proj = 10240 if C == 3 else 2048
    dft = 17 * 64 if C == 3 else 0
    fibres = 64 * C
    return K * 2 * (proj + dft) + 2 * 4 * (K - 1) * fibres + K * fibres


# ------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"htsvd_bench_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------- CPU oracle
#
# The FP64 oracle, as it stands, on all host cores: a spawn pool of single-threaded workers. Per image
# the fixed costs (noise estimate where sigma is estimated, global bases) are paid once; the groups
# are sampled by whole reference rows spread over each image, and the full-image time is projected
# as fixed-cost wall time + sampled-row wall time x (all rows / sampled rows).

_OW = {}


def _oracle_images(workload: str):
    """(noisy uint8 image, sigma or None = estimated, params) of every image of one step."""
    from paper_2508_10307_gb300 import synth
    if workload == "rgb4k":
        clean = synth.clean_image(2160, 3840, 3, 1003)
        prm = dict(ps=8, stride=3, window=31, K=32)
        return [(synth.add_poisson_gaussian(clean, 0.01, b * b, 1003), b, prm) for b in (10.0, 25.0, 50.0)]
    if workload == "rgb512":
        _, noisy, _, prm = synth.workload_rgb512()
        return [(noisy, None, prm)]
    raise ValueError(f"no CPU baseline for workload {workload}")


def _ow_init(workload: str):
    _OW["imgs"] = _oracle_images(workload)


def _ow_fixed(j: int):
    from oracle import htsvd_oracle as O
    noisy, sigma, prm = _OW["imgs"][j]
    p = O.Params.of(prm)
    t0 = time.perf_counter()
    if sigma is None:
        sigma = O.estimate_sigma(noisy, p)
    basis = O.global_basis(O.reference_patches(noisy, p))
    return sigma, basis, time.perf_counter() - t0


def _ow_rows(task):
    import numpy as np
    from oracle import htsvd_oracle as O
    j, rows, sigma, basis = task
    noisy, _, prm = _OW["imgs"][j]
    p = O.Params.of(prm)
    xs = O.reference_positions(noisy.shape[1], p.ps, p.stride)
    t0 = time.perf_counter()
    idx = np.concatenate([O._match_row(noisy, int(ry), xs, p)[0] for ry in rows])
    with np.errstate(divide="ignore", invalid="ignore"):     # pixels outside the sampled groups: 0 / 0
        O.denoise(noisy, sigma, p, idx=idx, basis=basis)
    return len(idx), time.perf_counter() - t0


class OraclePool:
    """All host cores running the oracle on one workload (spawned workers, one thread each)."""

    def __init__(self, workload: str):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.cores = len(os.sched_getaffinity(0))
        self.workload = workload
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_ow_init, initargs=(workload,))
        self.meta = [(x.shape, prm) for x, _, prm in _oracle_images(workload)]

    def fixed(self):
        """Per-image fixed costs, all images at once; returns the wall seconds."""
        t0 = time.perf_counter()
        self.fx = self.pool.map(_ow_fixed, range(len(self.meta)))
        return time.perf_counter() - t0

    def rows(self, per_image: int, offset: int = 0):
        """Wall seconds of per_image evenly spread reference rows of every image (two rows per task),
        the rows sampled and the rows in all; offset shifts the sample between calls."""
        from oracle import htsvd_oracle as O
        tasks, sampled, total = [], 0, 0
        for j, ((Hh, Ww, C), prm) in enumerate(self.meta):
            p = O.Params.of(prm)
            ys = O.reference_positions(Hh, p.ps, p.stride)
            total += len(ys)
            pick = [ys[(offset + (i * len(ys)) // per_image) % len(ys)] for i in range(per_image)]
            sampled += len(pick)
            for k in range(0, len(pick), 2):
                tasks.append((j, pick[k:k + 2], self.fx[j][0], self.fx[j][1]))
        t0 = time.perf_counter()
        self.pool.map(_ow_rows, tasks, chunksize=1)
        return time.perf_counter() - t0, sampled, total

    def close(self):
        self.pool.terminate()


def cpu_baseline(workload: str, mp_per_step: float) -> dict:
    """The oracle's projected whole-workload throughput on all host cores (bounded sample)."""
    op = OraclePool(workload)
    try:
        t_fixed = op.fixed()
        per_image = max(4, (2 * op.cores) // len(op.meta))
        t_rows, sampled, total = op.rows(per_image)
    finally:
        op.close()
    proj = t_fixed + t_rows * total / sampled
    return {"value": mp_per_step / proj, "unit": UNIT, "cores": op.cores, "kind": "oracle",
            "sample": f"{sampled} of {total} reference rows spread over the {len(op.meta)} image(s) of one step "
                      f"({t_rows:.1f} s), per-image noise estimate and bases once ({t_fixed:.1f} s); full-step "
                      f"time projected as {t_fixed:.1f} + {t_rows:.1f} x {total}/{sampled} = {proj:.0f} s"}


# The MRI workload's oracle baseline: the volume's bases once (timed, the fixed cost), then whole planes
# of references (one z index of the reference grid each) spread over the grid, grouped and filtered by
# single-threaded workers; the volume's time is projected as fixed + sampled-plane wall x planes / sampled.

def _mri_volume():
    from paper_2508_10307_gb300 import synth
    return synth.add_gaussian(synth.clean_volume(176, 208, 176, 3), 11.5, 3)


def _ov_init(basis):
    from oracle import htsvd_oracle as O
    _OW["vol"], _OW["vprm"], _OW["vbasis"] = _mri_volume(), O.Params.of(dict(ps=4, stride=2, window=5, K=32)), basis


def _ov_plane(iz):
    import numpy as np
    from oracle import htsvd_oracle as O
    v, p = _OW["vol"], _OW["vprm"]
    ny, nx = (len(O.reference_positions(n, p.ps, p.stride)) for n in v.shape[1:])
    t0 = time.perf_counter()
    idx = O.block_match_volume(v, p, only=np.arange(iz * ny * nx, (iz + 1) * ny * nx))
    with np.errstate(divide="ignore", invalid="ignore"):      # voxels outside the sampled groups: 0 / 0
        O.denoise_volume(v, 11.5, p, idx=idx, basis=_OW["vbasis"])
    return time.perf_counter() - t0


def cpu_baseline_volume(mp_per_step: float) -> dict:
    """The oracle's projected throughput on the MRI workload on all host cores (bounded sample)."""
    import multiprocessing as mp
    from oracle import htsvd_oracle as O
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    cores = len(os.sched_getaffinity(0))
    vol = _mri_volume()
    p = O.Params.of(dict(ps=4, stride=2, window=5, K=32))
    t0 = time.perf_counter()
    basis = O.global_basis(O.gather_cubes(vol, O.volume_reference_positions(vol.shape, p), p.ps))
    t_fixed = time.perf_counter() - t0
    nz = len(O.reference_positions(176, 4, 2))
    pool = mp.get_context("spawn").Pool(cores, initializer=_ov_init, initargs=(basis,))
    try:
        pool.map(_ov_fixed_ready, range(cores), chunksize=1)     # every worker has built its volume
        planes = [(i * nz) // cores for i in range(cores)]
        t0 = time.perf_counter()
        pool.map(_ov_plane, planes, chunksize=1)
        t_planes = time.perf_counter() - t0
    finally:
        pool.terminate()
    proj = t_fixed + t_planes * nz / len(planes)
    return {"value": mp_per_step / proj, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(planes)} of {nz} planes of references (grouping and filter, {t_planes:.1f} s), the "
                      f"volume's bases once ({t_fixed:.1f} s); the volume's time projected as {t_fixed:.1f} + "
                      f"{t_planes:.1f} x {nz}/{len(planes)} = {proj:.0f} s"}


def _ov_fixed_ready(_):
    return "vol" in _OW


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = args.workload if args.workload in ("rgb4k", "rgb512") else "rgb4k"
    mp_step = {"rgb4k": 3 * 3840 * 2160 / 1e6, "rgb512": 512 * 512 / 1e6}[wl]
    op = OraclePool(wl)
    try:
        t_fixed = op.fixed()                       # per-image fixed costs, measured once, charged every step
        per_image = max(2, op.cores // len(op.meta))
        for w in range(args.warmup):
            op.rows(per_image, offset=w)
        secs, samp, tot = 0.0, 0, 0
        for k in range(args.steps):
            t, samp, tot = op.rows(per_image, offset=args.warmup + k)
            secs += t_fixed + t * tot / samp
    finally:
        op.close()
    value = args.steps * mp_step / secs
    sample = (f"per step {samp} of {tot} reference rows spread over the image(s) of the {wl} workload on "
              f"{op.cores} cores, projected to the whole step; per-image noise estimate and bases measured "
              f"once ({t_fixed:.1f} s) and charged to every step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": op.cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------------------------------- GPU arm

def max_over_ranks_ms(ms, dist=None) -> float:
    """The slowest rank's time: whole-job throughput divides all ranks' work by it."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, steps: int, mp_per_step: float, max_ms: float) -> float:
    """Megapixels of every rank's steps over the slowest rank's device time (weak scaling)."""
    return world * steps * mp_per_step / (max_ms / 1000.0)


class Workload:
    """One bench step: inputs resident on the device, the call a user makes, the result it returns."""

    def __init__(self, name, config, mp_per_step, groups_per_step, C, K, host_inputs, step, result_bytes,
                 compare=None, compare_name=None, per_input=None):
        self.name, self.config, self.mp_per_step = name, config, mp_per_step
        self.groups_per_step, self.C, self.K = groups_per_step, C, K
        self.host_inputs, self.step, self.result_bytes = host_inputs, step, result_bytes
        self.compare, self.compare_name = compare, compare_name
        # independent calls, one per input (the step is their list): end to end, input i+1's copy in
        # and output i's copy out then overlap the calls on their own streams
        self.per_input = per_input


def volume_adaptive_groups(shape, sub, ps, stride):
    """Reference cubes over all sub-volumes of the adaptive volume call: per part and axis the grid
    {0, s, 2s, ...} plus the last position n - ps."""
    from paper_2508_10307_gb300 import subimage_bounds

    def grid(n):
        return len(range(0, n - ps + 1, stride)) + (1 if (n - ps) % stride else 0)

    total = 0
    for z0, z1 in subimage_bounds(shape[0], sub[0]):
        for y0, y1 in subimage_bounds(shape[1], sub[1]):
            for x0, x1 in subimage_bounds(shape[2], sub[2]):
                total += grid(z1 - z0) * grid(y1 - y0) * grid(x1 - x0)
    return total


def make_workload(name):
    import numpy as np
    import torch
    import paper_2508_10307_gb300 as H
    from paper_2508_10307_gb300 import synth

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    if name == "rgb512":
        clean, noisy, _, prm = synth.workload_rgb512()
        host = [noisy]
        n = H.num_groups(512, 512, prm)
        return Workload(name, workload_config("rgb512"), 512 * 512 / 1e6, n, 3, 32, host,
                        lambda d: [H.denoise(d[0], None, prm)], 512 * 512 * 3 * 4), clean
    if name == "gray128":
        clean, noisy, sigma, prm = synth.workload_gray128()
        cfg = {"workload": "gray128_sigma25", "image": "128x128x1 uint8", "noise": "gaussian sigma=25",
               "sigma": "given (25)", "ps": 8, "stride": 3, "window": 21, "K": 16, "tau": "2.7 sigma"}
        return Workload(name, cfg, 128 * 128 / 1e6, H.num_groups(128, 128, prm), 1, 16, [noisy],
                        lambda d: [H.denoise(d[0], sigma, prm)], 128 * 128 * 4), clean
    if name == "rgb4k":
        clean = synth.clean_image(2160, 3840, 3, 1003)
        levels = [10.0, 25.0, 50.0]
        noisy = [synth.add_poisson_gaussian(clean, 0.01, b * b, 1003) for b in levels]
        prm = dict(ps=8, stride=3, window=31, K=32)
        n = H.num_groups(2160, 3840, prm)
        calls = [(lambda x, b=b: H.denoise(x, b, prm)) for b in levels]
        return Workload(name, workload_config("rgb4k"), 3 * 3840 * 2160 / 1e6, 3 * n, 3, 32, noisy,
                        lambda d: [f(x) for f, x in zip(calls, d)],
                        3 * 3840 * 2160 * 3 * 4, per_input=calls), synth.quantize(clean)
    if name == "rgb1080":
        # one image of the headline's geometry at a quarter of its size: the small case that ncu captures
        clean = synth.clean_image(1080, 1920, 3, 1003)
        noisy = synth.add_poisson_gaussian(clean, 0.01, 25.0 ** 2, 1003)
        prm = dict(ps=8, stride=3, window=31, K=32)
        cfg = {"workload": "rgb1920x1080_pg_b625", "image": "1920x1080x3 uint8", "noise": "poisson-gaussian a=0.01 b=25^2",
               "sigma": "given (25)", "ps": 8, "stride": 3, "window": 31, "K": 32,
               "groups_per_image": H.num_groups(1080, 1920, prm)}
        return Workload(name, cfg, 1920 * 1080 / 1e6, H.num_groups(1080, 1920, prm), 3, 32, [noisy],
                        lambda d: [H.denoise(d[0], 25.0, prm)], 1920 * 1080 * 3 * 4), synth.quantize(clean)
    if name == "hsi696":
        # a 696 x 520 x 34 cube, the size of the paper's real-world HSI scenes (Sec. IV)
        clean = synth.clean_cube(520, 696, 34, 6001)
        noisy = synth.add_gaussian(clean, 12.0, 6001)
        prm = dict(ps=8, stride=3, window=18, K=32)
        cfg = {"workload": "hsi_696x520x34", "cube": "520x696x34 uint8 (three endmember spectra, smooth abundances)",
               "noise": "gaussian sigma=12", "sigma": "given (12)", "ps": 8, "stride": 3, "window": 18, "K": 32,
               "form": "Alg. 1 with the t-SVD along the band mode (34 Fourier slices), SSD over all bands"}
        n = H.num_groups(520, 696, prm)
        return Workload(name, cfg, 520 * 696 / 1e6, n, 34, 32, [noisy],
                        lambda d: [H.denoise_cube(d[0], 12.0, prm)], 520 * 696 * 34 * 4), synth.quantize(clean)
    if name == "batch64":
        shapes = synth.batch_shapes(64)
        imgs, sig, cleans = [], [], []
        for j, (h, w, s_) in enumerate(shapes):
            c, n_ = synth.batch_image(j, h, w, s_)
            imgs.append(n_)
            sig.append(s_)
        prm = dict(ps=8, stride=3, window=31, K=32)
        mp = sum(h * w for h, w, _ in shapes) / 1e6
        groups = sum(H.num_groups(h, w, prm) for h, w, _ in shapes)
        outs = [None]
        cfg = {"workload": "batch64_rgb_uneven", "images": "64 RGB uint8, W~U{256..2048}, H~U{256..1536}",
               "noise": "gaussian, sigma_j~U(10,50)", "sigma": "given per image", "ps": 8, "stride": 3,
               "window": 31, "K": 32, "form": "one persistent launch per phase, CUDA graph replay, autotuned tiles"}

        def step(d):
            if outs[0] is None:
                outs[0] = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in d]
            return H.denoise_batch(d, sig, prm, outs=outs[0])

        def sequential(d):
            return [H.denoise(x, s_, prm) for x, s_ in zip(d, sig)]

        return Workload(name, cfg, mp, groups, 3, 32, imgs, step, int(mp * 1e6 * 12), sequential,
                        "sequential_plain_calls"), None
    if name == "vjp8":
        cleans, xs = [], []
        for j in range(8):
            c = synth.clean_image(512, 512, 3, 3000 + j)
            cleans.append(c.astype(np.float32))
            xs.append(synth.add_gaussian_float(c, 25.0, 3000 + j))
        prm = dict(ps=8, stride=2, window=31, K=32)
        n = H.num_groups(512, 512, prm)
        targets = [None]
        cfg = {"workload": "vjp8_rgb512_f32", "images": "8 x 512x512x3 float32", "noise": "gaussian sigma=25",
               "sigma": "given (25)", "ps": 8, "stride": 2, "window": 31, "K": 32,
               "form": "forward + hand-written VJP (x and per-group weights), loss = MSE to the clean image"}

        def step(d):
            if targets[0] is None:
                targets[0] = [dev(c) for c in cleans]
            res = []
            for x, t in zip(d, targets[0]):
                xr = x.detach().requires_grad_(True)
                w = torch.ones(n, device="cuda", requires_grad=True)
                out = H.HtsvdFn.apply(xr, w, 25.0, prm)
                loss = ((out - t) ** 2).mean()
                loss.backward()
                res.append(xr.grad)
            return res

        def forward_only(d):
            return [H.denoise_f32(x, 25.0, prm) for x in d]

        return Workload(name, cfg, 8 * 512 * 512 / 1e6, 8 * n, 3, 32, xs, step, 8 * 512 * 512 * 3 * 4,
                        forward_only, "forward_only"), None
    if name in ("mri176", "mri176est"):
        # an MRI-sized volume (the OASIS T1-weighted grid, 176 x 208 x 176) at the paper's MRI setting;
        # mri176est estimates sigma from the reference cubes' covariance eigenvalues
        clean = synth.clean_volume(176, 208, 176, 3)
        noisy = synth.add_gaussian(clean, 11.5, 3)
        prm = dict(ps=4, stride=2, window=5, K=32)
        n = 87 * 103 * 87
        est = name == "mri176est"
        cfg = {"workload": "mri_volume_176x208x176" + ("_sigma_est" if est else ""),
               "volume": "176x208x176 uint8 (head-like phantom)",
               "noise": "gaussian sigma=11.5 (4.5% of 255; stands in for VST-stabilised Rician noise)",
               "sigma": "estimated (cube-covariance eigenvalues)" if est else "given", "ps": "4x4x4", "stride": 2,
               "window": "5x5x5", "K": 32, "unit_note": "MP/s counts voxels (D H W) as pixels"}

        def step(d):
            return [H.denoise_volume(x, None if est else 11.5, prm) for x in d]

        return Workload(name, cfg, 176 * 208 * 176 / 1e6, n, 4, 32, [noisy], step, 176 * 208 * 176 * 4), \
            synth.quantize(clean)
    if name == "mri176adapt":
        # the adaptive variant (Alg. 2) on the MRI-sized volume: 2 x 2 x 2 sub-volumes of 88 x 104 x 88, a
        # sigma per sub-volume from its reference cubes' covariance eigenvalues, each part denoised on its own
        clean = synth.clean_volume(176, 208, 176, 3)
        noisy = synth.add_gaussian(clean, 11.5, 3)
        prm = dict(ps=4, stride=2, window=5, K=32)
        sub = (88, 104, 88)
        n = volume_adaptive_groups((176, 208, 176), sub, 4, 2)
        cfg = {"workload": "mri_volume_176x208x176_adaptive_2x2x2",
               "volume": "176x208x176 uint8 (head-like phantom)",
               "noise": "gaussian sigma=11.5 (4.5% of 255; stands in for VST-stabilised Rician noise)",
               "sigma": "estimated per sub-volume (cube-covariance eigenvalues)", "sub_volume": "88x104x88",
               "ps": "4x4x4", "stride": 2, "window": "5x5x5", "K": 32,
               "unit_note": "MP/s counts voxels (D H W) as pixels"}

        def step(d):
            return [H.denoise_volume_adaptive(x, sub, prm) for x in d]

        return Workload(name, cfg, 176 * 208 * 176 / 1e6, n, 4, 32, [noisy], step, 176 * 208 * 176 * 4), \
            synth.quantize(clean)
    if name == "proj512all":
        # the batched basis projection of every patch position of the 512x512x3 image (505 x 505 =
        # 255,025 patches, an im2col batch), tensor cores against the structured FP32 form
        clean, noisy, _, prm = synth.workload_rgb512()
        setup = {}
        cfg = {"workload": "projection_rgb512_every_position", "image": "512x512x3 uint8",
               "noise": "poisson-gaussian a=0.01 b=15^2", "patches_per_step": 505 * 505,
               "form": "S = U^T * P * V of every 8x8x3 patch position (192 FP32 coefficients each), tensor cores: "
                       "dense 192x192 contraction, matrix split in two FP16 pieces, im2col tiles"}

        def prepare(x):
            if "basis" not in setup:
                _, info = H.denoise(x, None, prm, return_info=True, basis=True)
                setup["basis"] = info["basis"].reshape(-1).contiguous()
                setup["out"] = torch.empty((505 * 505, 192), dtype=torch.float32, device="cuda")
            return setup

        def step(d):
            st = prepare(d[0])
            return [H.project_patches(d[0], None, st["basis"], out=st["out"])]

        def structured(d):
            st = prepare(d[0])
            return [H.project_patches(d[0], None, st["basis"], out=st["out"], structured=True)]

        return Workload(name, cfg, 512 * 512 / 1e6, 505 * 505, 3, 1, [noisy], step, 505 * 505 * 192 * 4,
                        structured, "structured_fp32_cuda_cores"), None
    if name == "proj512":
        # the batched basis projection of every patch of every group of the 512x512x3 workload (64,009
        # groups x 32 members), on the tensor cores; compared with the structured FP32 form on the CUDA cores
        clean, noisy, _, prm = synth.workload_rgb512()
        setup = {}
        cfg = {"workload": "projection_rgb512_members", "image": "512x512x3 uint8",
               "noise": "poisson-gaussian a=0.01 b=15^2", "ps": 8, "stride": 2, "window": 31, "K": 32,
               "patches_per_step": 64009 * 32,
               "form": "S = U^T * P * V of every group member (64,009 x 32 patches, 192 FP32 coefficients each), "
                       "tensor cores: dense 192x192 contraction, matrix split in two FP16 pieces"}

        def prepare(x):
            if "pos" not in setup:
                _, info = H.denoise(x, None, prm, return_info=True, basis=True)
                setup["pos"] = info["idx"].reshape(-1).contiguous()
                setup["basis"] = info["basis"].reshape(-1).contiguous()
                setup["out"] = torch.empty((setup["pos"].numel(), 192), dtype=torch.float32, device="cuda")
            return setup

        def step(d):
            st = prepare(d[0])
            return [H.project_patches(d[0], st["pos"], st["basis"], out=st["out"])]

        def structured(d):
            st = prepare(d[0])
            return [H.project_patches(d[0], st["pos"], st["basis"], out=st["out"], structured=True)]

        return Workload(name, cfg, 512 * 512 / 1e6, 64009, 3, 32, [noisy], step, 64009 * 32 * 192 * 4,
                        structured, "structured_fp32_cuda_cores"), None
    if name == "adaptive512":
        clean, noisy, _, prm = synth.workload_rgb512()
        prm = dict(prm, adapt=True)
        sub = (256, 256)
        cfg = {"workload": "a_haar_tsvd_rgb512_sub256", "image": "512x512x3 uint8",
               "noise": "poisson-gaussian a=0.01 b=15^2", "subimages": "2 x 2 of 256x256",
               "sigma": "estimated per subimage (eigenvalue rule + eigen-rank vote)", "ps": 8, "stride": 2,
               "window": 31, "K": 32, "form": "Alg. 2: one host sync, subimages denoised as one batch"}
        n = H.num_groups(256, 256, prm) * 4

        def plain(d):
            return [H.denoise(d[0], None, dict(prm, adapt=False))]

        return Workload(name, cfg, 512 * 512 / 1e6, n, 3, 32, [noisy],
                        lambda d: [H.denoise_adaptive(d[0], sub, prm)], 512 * 512 * 3 * 4, plain,
                        "plain_single_sigma"), clean
    if name == "video1080":
        F, Hh, Ww, T = 4, 1080, 1920, 1
        base = synth.clean_image(Hh, Ww + F, 3, 4001)
        clip = np.stack([synth.add_poisson_gaussian(np.ascontiguousarray(base[:, t:t + Ww]), 0.01, 15.0 ** 2,
                                                    4001 + 17 * t) for t in range(F)])
        prm = dict(ps=8, stride=3, window=31, K=32)
        cfg = {"workload": "video_rgb1920x1080x4_T1", "clip": "4 frames of 1920x1080x3 uint8, content drifting "
               "one pixel per frame", "noise": "poisson-gaussian a=0.01 b=15^2, fresh per frame",
               "sigma": "estimated per frame", "ps": 8, "stride": 3, "window": 31, "K": 32,
               "temporal_radius": T, "form": "frame by frame, grouping over frames t-1..t+1"}
        n = H.num_groups(Hh, Ww, prm)

        def frame_by_frame(d):
            return [H.denoise_video(d[0], None, prm, T=0)]

        clean = np.stack([synth.quantize(base[:, t:t + Ww]) for t in range(F)])
        return Workload(name, cfg, F * Hh * Ww / 1e6, F * n, 3, 32, [clip],
                        lambda d: [H.denoise_video(d[0], None, prm, T=T)], F * Hh * Ww * 3 * 4, frame_by_frame,
                        "frame_by_frame_no_temporal_search"), clean
    if name == "sweep512":
        clean, noisy, _, prm = synth.workload_rgb512()
        mults = [1.8, 2.1, 2.4, 2.7, 3.0, 3.3, 3.6, 3.9]
        cfg = {"workload": "tau_sweep_rgb512_x8", "image": "512x512x3 uint8", "noise": "poisson-gaussian a=0.01 b=15^2",
               "sigma": "estimated once", "tau_mults": mults, "ps": 8, "stride": 2, "window": 31, "K": 32,
               "form": "grouping, bases, sigma and noisy coefficients once; threshold, synthesis and aggregation "
                       "per tau (the step's MP count is 8 outputs)"}
        n = H.num_groups(512, 512, prm)
        sig = [None]

        def plain(d):
            if sig[0] is None:
                sig[0] = H.estimate_sigma(d[0], prm)
            return [H.denoise(d[0], sig[0], dict(prm, tau_mult=m)) for m in mults]

        return Workload(name, cfg, len(mults) * 512 * 512 / 1e6, len(mults) * n, 3, 32, [noisy],
                        lambda d: [H.denoise_tau_sweep(d[0], mults, None, prm)], len(mults) * 512 * 512 * 3 * 4,
                        plain, "separate_calls_per_tau"), None
    if name == "sure512":
        clean = synth.clean_image(512, 512, 3, 5001)
        y = synth.add_gaussian_float(clean, 25.0, 5001).astype(np.float32)
        probe = np.random.default_rng(5002).choice([-1.0, 1.0], size=y.shape).astype(np.float32)
        prm = dict(ps=8, stride=2, window=31, K=32)
        mults = [1.8, 2.4, 3.0, 3.6]
        cfg = {"workload": "sure_rgb512_f32_x4", "image": "512x512x3 float32", "noise": "gaussian sigma=25",
               "sigma": "given (25)", "tau_mults": mults, "ps": 8, "stride": 2, "window": 31, "K": 32,
               "form": "finite-difference divergence along a +-1 probe, eps = sigma/10: grouping and bases of y and of "
                       "y + eps probe once each, two forward passes per multiplier, FP64 sums (MP count: 4 images)"}
        n = H.num_groups(512, 512, prm)
        pb = [None]

        def step(d):
            if pb[0] is None:
                pb[0] = dev(probe)
            return [torch.tensor(H.sure(d[0], 25.0, mults, pb[0], prm))]

        def forward_only(d):
            return [H.denoise_f32(d[0], 25.0, dict(prm, tau_mult=m)) for m in mults]

        return Workload(name, cfg, len(mults) * 512 * 512 / 1e6, len(mults) * n, 3, 32, [y], step, 8 * len(mults),
                        forward_only, "forward_only_per_tau"), None
    if name == "tunew512":
        clean = synth.clean_image(512, 512, 3, 5101)
        y = synth.add_gaussian_float(clean, 25.0, 5101).astype(np.float32)
        probe = np.random.default_rng(5102).choice([-1.0, 1.0], size=y.shape).astype(np.float32)
        prm = dict(ps=8, stride=3, window=31, K=32)
        steps = 4
        cfg = {"workload": "tune_weights_rgb512_f32", "image": "512x512x3 float32", "noise": "gaussian sigma=25",
               "sigma": "given (25)", "ps": 8, "stride": 3, "window": 31, "K": 32, "steps": steps, "step": 0.5,
               "form": "per-group weights tuned by exponentiated-gradient steps on their SURE (eps = sigma/10): "
                       "grouping and bases of y and y + eps probe once, per step two forward passes and two VJPs "
                       "(MP count: one image per SURE evaluation)"}
        n = H.num_groups(512, 512, prm)
        pb = [None]
        trace = [None]

        def step(d):
            if pb[0] is None:
                pb[0] = dev(probe)
            w, tr = H.tune_weights(d[0], 25.0, pb[0], prm, eps=2.5, steps=steps, step=0.5)
            trace[0] = tr
            return [w]

        def forward_only(d):
            return [H.denoise_f32(d[0], 25.0, prm)]

        return Workload(name, cfg, (steps + 1) * 512 * 512 / 1e6, (steps + 1) * n, 3, 32, [y], step, 4 * n,
                        forward_only, "forward_only"), None
    raise ValueError(name)


def run_gpu(args):
    import torch
    import paper_2508_10307_gb300 as H
    from paper_2508_10307_gb300 import _lib, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    H.load_library()
    wl, clean = make_workload(args.workload)
    d_in = [torch.from_numpy(x).cuda() for x in wl.host_inputs]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # warm-up (also grows the workspace, tunes and captures the batch graph)
    for _ in range(args.warmup):
        res = wl.step(d_in)
    torch.cuda.synchronize()
    psnr_gpu = synth.psnr(res[0].detach().cpu().numpy(), clean) if clean is not None else None

    def timed(fn, inputs_dev, steps, with_copies=False, hosts=None, host_out=None):
        evs = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if with_copies:
                for hsrc, ddst in zip(hosts, inputs_dev):
                    ddst.copy_(hsrc, non_blocking=True)
            r = fn(inputs_dev)
            if with_copies:
                for ro, ho in zip(r, host_out):
                    ho.copy_(ro.detach(), non_blocking=True)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()

    def timed_pipelined(calls, inputs_dev, steps, hosts, host_out):
        """End to end with the copies overlapped: input i copied in on one stream, call i on the
        compute stream once it has arrived, output i copied out on another stream once call i is
        done; the end event waits for the last copy out. Every copy stays inside the timed region."""
        evs = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            copy_in.wait_event(a)
            arrived = []
            for hsrc, ddst in zip(hosts, inputs_dev):
                with torch.cuda.stream(copy_in):
                    ddst.copy_(hsrc, non_blocking=True)
                    e = torch.cuda.Event()
                    e.record(copy_in)
                arrived.append(e)
            for f, x, e, ho in zip(calls, inputs_dev, arrived, host_out):
                stream.wait_event(e)
                r = f(x)
                done = torch.cuda.Event()
                done.record(stream)
                copy_out.wait_event(done)
                with torch.cuda.stream(copy_out):
                    r.record_stream(copy_out)
                    ho.copy_(r.detach(), non_blocking=True)
            stream.wait_stream(copy_out)
            stream.wait_stream(copy_in)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    def max_over_ranks(ms):
        return max_over_ranks_ms(ms, dist)

    sampler = ClockSampler(local)
    _lib.profile_enable(True)
    _lib.profile_collect()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    dev_ms = timed(wl.step, d_in, args.steps)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    prof = _lib.profile_collect()
    _lib.profile_enable(False)
    host_steps = {k: v for k, v in prof.items() if k.endswith("_host")}     # wall-clock host steps, not launches
    prof = {k: v for k, v in prof.items() if k not in host_steps}
    dev_ms_max = max_over_ranks(dev_ms)
    value = whole_job_value(world, args.steps, wl.mp_per_step, dev_ms_max)

    # end to end through the public API: pinned host inputs -> device, the call, results -> pinned host
    hosts = [torch.from_numpy(x).pin_memory() for x in wl.host_inputs]
    res = wl.step(d_in)
    host_out = [torch.empty(r.shape, dtype=r.dtype).pin_memory() for r in res]
    if wl.per_input is not None:
        timed_pipelined(wl.per_input, d_in, args.warmup, hosts, host_out)
        e2e_ms = max_over_ranks(timed_pipelined(wl.per_input, d_in, args.steps, hosts, host_out))
    else:
        timed(wl.step, d_in, args.warmup, True, hosts, host_out)
        e2e_ms = max_over_ranks(timed(wl.step, d_in, args.steps, True, hosts, host_out))
    e2e_value = whole_job_value(world, args.steps, wl.mp_per_step, e2e_ms)
    h2d = sum(x.nbytes for x in wl.host_inputs)
    d2h = sum(h.numel() * h.element_size() for h in host_out)

    compare = None
    if wl.compare is not None:
        for _ in range(args.warmup):
            wl.compare(d_in)
        cmp_ms = max_over_ranks(timed(wl.compare, d_in, args.steps))
        cmp_value = whole_job_value(world, args.steps, wl.mp_per_step, cmp_ms)
        compare = {"name": wl.compare_name, "value": cmp_value, "unit": UNIT, "ms_per_step": cmp_ms / args.steps,
                   "ratio": value / cmp_value}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (by device time in the timed region)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    launches = sum(v[0] for v in prof.values()) if prof else 5 * args.steps
    roof = None
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    probe = {name: float(_lib.load().htsvd_internal_alu_probe(op, 2048)) for op, name in
             ((0, "ffma"), (1, "imad"), (2, "dp4a"))}
    if dom == "filter":
        n_launch, ms = prof["filter"]
        flops = wl.groups_per_step * filter_flops_per_group(wl.C, wl.K) * args.steps / n_launch
        achieved = flops / (ms / n_launch / 1000.0) / 1e12
        peak = nsm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": FILTER_DRAM_BYTES.get(args.workload), "kernel": "group_filter",
                "peak_basis": f"FP32 FMA: {nsm} SMs (device query) x {FP32_LANES_PER_SM} lanes x 2 flop x "
                              f"{MAX_SM_MHZ:.0f} MHz (unit counts and max clock); issue-rate probe in this run: "
                              f"{probe['ffma']:.1f} FFMA, {probe['imad']:.1f} IMAD, {probe['dp4a']:.1f} DP4A per SM clock"}
    elif dom == "cube_filter":
        # forward transforms of every Haar slot as the kernel computes them (the inverse of the slots that
        # keep a coefficient depends on the data and is not counted): folded band DFT and its inverse,
        # 64 nf^2 MACs each for the real and the imaginary part, and two per-slice 8x8 complex products
        n_launch, ms = prof["cube_filter"]
        nf = wl.C // 2 + 1
        flops = wl.groups_per_step * wl.K * 2 * (256 * nf * nf + 4096 * nf) * args.steps / n_launch
        achieved = flops / (ms / n_launch / 1000.0) / 1e12
        peak = nsm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "cube_filter",
                "peak_basis": f"FP32 FMA: {nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {MAX_SM_MHZ:.0f} MHz; "
                              "achieved counts the forward transforms only"}
    elif dom == "volume_filter":
        n_launch, ms = prof["volume_filter"]
        flops = wl.groups_per_step * volume_flops_per_group(wl.K) * args.steps / n_launch
        achieved = flops / (ms / n_launch / 1000.0) / 1e12
        peak = nsm * FP32_LANES_PER_SM * 2 * MAX_SM_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "volume_filter",
                "peak_basis": f"FP32 FMA: {nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {MAX_SM_MHZ:.0f} MHz"}
    elif dom == "project_tc":
        # the dense contraction as the algorithm of this kernel: 2 (64 C)^2 flop per patch (two FP16
        # products of it execute); peak: the measured BF16 dense rate (FP16 has the same nominal rate)
        n_launch, ms = prof["project_tc"]
        patches = wl.groups_per_step * wl.K
        flops = 2.0 * (64 * wl.C) ** 2 * patches * args.steps / n_launch
        achieved = flops / (ms / n_launch / 1000.0) / 1e12
        peak = measured_peak("bf16_tflops")
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": None, "kernel": "project_tc",
                "executed_tflops": 2 * achieved,
                "out_gbs": patches * 64 * wl.C * 4 * args.steps / n_launch / (ms / n_launch / 1000.0) / 1e9,
                "peak_basis": "dense BF16 cuBLAS burst, measured (MEASURED_PEAKS.json), times the nominal FP16/BF16 "
                              "ratio 1; achieved counts the dense contraction once (two FP16 pieces execute)"}
    elif dom is not None:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None,
                "kernel": dom}

    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload in ("rgb4k", "rgb512", "mri176"):
        try:
            cpu = (cpu_baseline_volume(wl.mp_per_step) if args.workload == "mri176"
                   else cpu_baseline(args.workload, wl.mp_per_step))
        except Exception as e:  # the baseline is reported, never allowed to sink the GPU number
            cpu = {"value": None, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                   "sample": f"failed: {e}"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(wl.config, l2="256 MB buffer written between timed steps (untimed)",
                           parallelism=f"replicas x{world}"),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "kernels_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
            "host_ms": {k: {"calls": v[0], "ms": v[1]} for k, v in host_steps.items()},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "psnr_db": psnr_gpu}
    if compare is not None:
        line["compare"] = compare
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rgb4k", choices=["rgb512", "gray128", "rgb4k", "rgb1080", "hsi696", "batch64", "vjp8", "adaptive512",
                                                      "video1080", "sweep512", "sure512", "tunew512", "proj512", "proj512all", "mri176", "mri176est",
                                                      "mri176adapt"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
