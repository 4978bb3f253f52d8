"""Benchmark: Gauss-Newton Hessian-vector products per second on one GB300.

Workload (the paper-scale configuration): 384 x 1152 interior grid at 8 m plus
a 40-cell sponge (464 x 1232 padded), seeded layered/faulted velocity model
1500-5500 m/s smoothed to the Gauss-Newton point, 32 Ricker shots at 10 Hz,
384 receivers every 24 m, 3000 steps at dt = 0.727 ms, binomial checkpointing
with 30 snapshots per shot.  One step = one H v (forward, Born and adjoint
sweeps over all 32 shots, recomputation from snapshots, imaging reduction).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line.  Under torchrun the one H v is split over the ranks
(strong scaling): each rank owns a contiguous block of the shots, computes the
extended image of its block in FP64 on the padded grid, the images are
gathered over NCCL and summed in rank order on every rank (the one exchange
step), and the sum is folded onto the interior once; the time is the maximum
over ranks.  --impl reference times the FP64 CPU oracle on a bounded sample
of the same workload on the host's cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·v/s and Gpt-updates/s (% HBM peak) at ≤2e-4 rel err vs FP64; serve p50/p99"

CKPT = 30
ENGINE_LOOP = False   # misfit lanes served by the engine's device-resident loop (--engine-loop)
UNIT = "H·v/s"


def workload_config(w):
    return {
        "workload": f"GN Hessian apply, {w.nz}x{w.nx} grid at {w.h:g} m + {w.nb}-cell sponge "
                    f"({w.nz + 2 * w.nb}x{w.nx + 2 * w.nb} padded), {w.ns} shots x {w.nr} receivers, "
                    f"{w.nt} steps, {w.k} vector{'s' if w.k > 1 else ''}, "
                    + (f"{CKPT} snapshots/shot (binomial checkpointing)" if CKPT > 0 else "every time level stored"),
        "grid": [w.nz, w.nx], "sponge": w.nb, "h_m": w.h, "shots": w.ns, "receivers": w.nr, "steps": w.nt,
        "dt_s": w.dt, "f0_hz": w.f0, "vectors": w.k, "snapshots_per_shot": CKPT,
        "l2": "inputs larger than L2 (per-step working set of fields and snapshots >> 129 MB)",
    }


# FP32 multiply-add rate of the part: 152 SMs x 128 FP32 lanes x 2.07 GHz.
FP32_FMA_PEAK = 152 * 128 * 2.07e9


def psf_fma_count(nz, nx, S, B):
    """Multiply-adds of one PSF apply: (2R+1)^2 per nonzero bilinear weight per point."""
    R = (B * S - 1) // 2
    c0 = S // 2

    def terms(n):
        na = (n - 1 - c0) // S + 1
        q = np.clip(np.arange(n) - c0, 0, (na - 1) * S)
        a0 = np.minimum(q // S, max(na - 2, 0))
        rem = q - a0 * S
        return np.where((rem > 0) & (rem < S), 2, 1)

    return int(np.outer(terms(nz), terms(nx)).sum()) * (2 * R + 1) ** 2


def pdo_measure(P, m, w, dev, r=8, reps=10):
    """Build time of the PDO approximation (one H v, cuFFT separation) and apply rate for the
    workload's vectors; rho0 = 2 pi f_max / c_max with f_max = 2.5 f0 (the appendix's choice)."""
    import torch

    from paper_2507_10804_gb300.hv import HV_CKPT_ALL
    rho0 = 2 * np.pi * 2.5 * w.f0 / float(w.vmax)
    st = torch.cuda.current_stream(dev)
    P.approx_build_pdo(m, rho0, r, ckpt=HV_CKPT_ALL).close()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    A = P.approx_build_pdo(m, rho0, r, ckpt=HV_CKPT_ALL)
    e1.record(st)
    torch.cuda.synchronize(dev)
    build_ms = e0.elapsed_time(e1)
    v = torch.tensor(w.v, dtype=torch.float32, device=dev)
    A.apply(v)
    torch.cuda.synchronize(dev)
    e0.record(st)
    for _ in range(reps):
        A.apply(v)
    e1.record(st)
    torch.cuda.synchronize(dev)
    apply_s = e0.elapsed_time(e1) / 1e3 / reps
    A.close()
    return {"rho0_rad_per_m": rho0, "terms": r, "build_ms": build_ms,
            "apply_us_per_vector": apply_s / v.shape[0] * 1e6, "apply_vectors_per_s": v.shape[0] / apply_s,
            "what": "per vector: one forward and r inverse complex 2D FFTs (cuFFT) and two fused pointwise kernels"}


def psfplus_measure(P, m, w, dev, S=12, n_batches=4, r=8, tol=1e-3, reps=10):
    """PSF+ from the workload's PSF and PDO approximations: combination time (rows, SVD, refinement)
    and apply rate."""
    import torch

    from paper_2507_10804_gb300.hv import HV_CKPT_ALL, psf_plus
    rho0 = 2 * np.pi * 2.5 * w.f0 / float(w.vmax)
    A = P.approx_build_psf(m, S, n_batches, ckpt=HV_CKPT_ALL)
    D = P.approx_build_pdo(m, rho0, r, ckpt=HV_CKPT_ALL)
    psf_plus(A, D, tol).close()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    C = psf_plus(A, D, tol)
    torch.cuda.synchronize(dev)
    build_ms = (time.perf_counter() - t0) * 1e3
    st = torch.cuda.current_stream(dev)
    v = torch.tensor(w.v, dtype=torch.float32, device=dev)
    C.apply(v)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        C.apply(v)
    e1.record(st)
    torch.cuda.synchronize(dev)
    apply_s = e0.elapsed_time(e1) / 1e3 / reps
    rank = C.info["r"]
    for x in (C, A, D):
        x.close()
    return {"rank": rank, "tol": tol, "combine_ms": build_ms, "apply_us_per_vector": apply_s / v.shape[0] * 1e6,
            "what": "combination of the PSF and PDO approximations above (host clock: includes the host "
                    "eigensolver); apply as the PDO one with rank terms"}


def lr_measure(P, m, w, dev, rank=16, k=24, delta=1.0, gamma=2500.0, reps=10):
    """Low-rank approximation with the Matern prior: build time (two batched H v of k vectors, the
    R-orthonormalisation and the host eigensolver) and apply rates of H~_d and of the sampling factor."""
    import torch

    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300.hv import HV_CKPT_ALL
    omega = torch.tensor(synth.normal(2025, k * w.nz * w.nx).reshape(k, w.nz, w.nx), dtype=torch.float32,
                         device=dev)
    P.approx_build_lr(m, delta, gamma, rank, omega, ckpt=HV_CKPT_ALL).close()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    A = P.approx_build_lr(m, delta, gamma, rank, omega, ckpt=HV_CKPT_ALL)
    torch.cuda.synchronize(dev)
    build_ms = (time.perf_counter() - t0) * 1e3
    v = torch.tensor(w.v, dtype=torch.float32, device=dev)
    res = {"rank": rank, "test_vectors": k, "delta": delta, "gamma": gamma, "build_ms": build_ms,
           "lambda_1": float(A.eigs()[0][0]), "lambda_r": float(A.eigs()[0][-1])}
    st = torch.cuda.current_stream(dev)
    for name, mode in (("apply_us_per_vector", 0), ("sample_us_per_vector", 2)):
        A.apply(v, mode)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            A.apply(v, mode)
        e1.record(st)
        torch.cuda.synchronize(dev)
        res[name] = e0.elapsed_time(e1) / 1e3 / reps / v.shape[0] * 1e6
    A.close()
    res["what"] = "build on the host clock (two batched H v); applies per vector, one vector per kernel chain"
    return res


def quad_measure(dev, nz=256, nx=256, h=10.0, chains=64, steps=10, warm=3, beta=0.5, delta=1.0, gamma=2500.0):
    """The quadratic test model: H_d apply rate, the square-root PSF+ approximation built through the
    operator interface, the corrected posterior (rank 32 of 40 test vectors), posterior samples by
    preconditioned CG, and gpCN steps of `chains` chains (sample, propose, objective, H~ apply, accept)."""
    import torch

    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300.hv import (Posterior, Quad, approx_build_pdo_op, approx_build_psf_op, gpcn_accept,
                                           gpcn_propose, psf_plus)
    lam = [40.0 * 0.8 ** j for j in range(10)]
    Q = Quad(nz, nx, h, lam, delta, gamma, device=dev)
    st = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    v = torch.tensor(synth.smoothed_normal_vectors(5, chains, nz, nx, 2.0), dtype=torch.float32, device=dev)
    Q.apply(v)
    torch.cuda.synchronize(dev)
    e0, e1 = ev(), ev()
    e0.record(st)
    for _ in range(5):
        Q.apply(v)
    e1.record(st)
    torch.cuda.synchronize(dev)
    hd_us = e0.elapsed_time(e1) / 5 / chains * 1e3
    t0 = time.perf_counter()
    A = approx_build_psf_op(Q, 16, 4)                  # 16 x 16 PSFs: PSF+ takes at most 256
    D = approx_build_pdo_op(Q, 0.08, 8)
    C = psf_plus(A, D, 1e-3, spd=True)
    post = Posterior(nz, nx, h, delta, gamma, approx=C)
    torch.cuda.synchronize(dev)
    build_ms = (time.perf_counter() - t0) * 1e3
    omega = torch.tensor(synth.normal(2026, 40 * nz * nx).reshape(40, nz, nx), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    post.correct(Q, omega, 32)
    torch.cuda.synchronize(dev)
    correct_ms = (time.perf_counter() - t0) * 1e3
    lam_c, _ = post.eigs()
    mstar = torch.tensor(synth.smoothed_normal_vectors(6, 1, nz, nx, 4.0)[0], dtype=torch.float32, device=dev)
    _, g0 = Q.objective(torch.zeros((1, nz, nx), device=dev), mstar)
    t0 = time.perf_counter()
    m_map, map_iters = post.solve(-g0, op=Q, rtol=1e-6)
    torch.cuda.synchronize(dev)
    map_ms = (time.perf_counter() - t0) * 1e3
    gen = torch.Generator(device=dev).manual_seed(11)
    m = m_map.repeat(chains, 1, 1).contiguous()
    phi, _ = Q.objective(m, mstar, grad=False)
    delta_cur = torch.empty(chains, dtype=torch.float64, device=dev)
    zero = torch.zeros_like(m)
    gpcn_accept(phi, m, zero, zero, torch.full((chains,), -float("inf"), dtype=torch.float64, device=dev), m,
                delta_cur)
    mp = m_map[0].contiguous()
    acc, iters = 0, []

    def step():
        nonlocal acc
        n1 = torch.randn((chains, nz, nx), device=dev, generator=gen)
        n2 = torch.randn((chains, nz, nx), device=dev, generator=gen)
        zeta, it = post.sample(n1, n2)
        iters.append(it)
        m_new, d_new = gpcn_propose(m, mp, zeta, beta)
        phi_new, _ = Q.objective(m_new, mstar, grad=False)
        Hd = post.apply(d_new)
        log_u = torch.log(torch.rand(chains, dtype=torch.float64, device=dev, generator=gen))
        return gpcn_accept(phi_new, m_new, d_new, Hd, log_u, m, delta_cur)

    for _ in range(warm):
        step()
    torch.cuda.synchronize(dev)
    iters.clear()
    accs = []
    t0 = time.perf_counter()
    for _ in range(steps):
        accs.append(step())
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    acc = float(torch.stack(accs).double().mean())
    res = {"grid": [nz, nx], "h_m": h, "lowrank_part": len(lam), "hd_apply_us_per_vector": hd_us,
           "psfplus_sqrt_rank": C.info["r"], "build_ms": build_ms, "correction_rank": 32, "correction_ms": correct_ms,
           "correction_lambda_1": float(lam_c[0]), "correction_lambda_r": float(lam_c[-1]),
           "map_solve_ms": map_ms, "map_cg_iterations": map_iters, "chains": chains, "beta": beta,
           "gpcn_steps_per_s": steps * chains / dt, "gpcn_ms_per_step": dt / steps * 1e3,
           "sample_cg_iterations": float(np.mean(iters)), "acceptance": acc,
           "what": "host clock around synchronised phases; a gpCN step advances every chain once"}
    for x in (post, C, D, A, Q):
        x.close()
    return res


def psf_measure(P, m, w, dev, S=12, n_batches=4, reps=10):
    """Build time of the PSF approximation (n_batches H v) and apply rate for the workload's vectors."""
    import torch

    from paper_2507_10804_gb300.hv import HV_CKPT_ALL
    st = torch.cuda.current_stream(dev)
    P.approx_build_psf(m, S, n_batches, ckpt=HV_CKPT_ALL).close()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    A = P.approx_build_psf(m, S, n_batches, ckpt=HV_CKPT_ALL)
    e1.record(st)
    torch.cuda.synchronize(dev)
    build_ms = e0.elapsed_time(e1)
    v = torch.tensor(w.v, dtype=torch.float32, device=dev)
    A.apply(v)
    torch.cuda.synchronize(dev)
    e0.record(st)
    for _ in range(reps):
        A.apply(v)
    e1.record(st)
    torch.cuda.synchronize(dev)
    apply_s = e0.elapsed_time(e1) / 1e3 / reps
    B = int(round(n_batches ** 0.5))
    fma = psf_fma_count(w.nz, w.nx, S, B) * v.shape[0]
    A.close()
    return {"spacing_cells": S, "batches": n_batches, "psfs": A.info["r"], "window_radius": A.info["R"],
            "build_ms": build_ms, "apply_us_per_vector": apply_s / v.shape[0] * 1e6,
            "apply_vectors_per_s": v.shape[0] / apply_s,
            "roofline": {"bound": "alu", "achieved": fma / apply_s / 1e12, "peak": FP32_FMA_PEAK / 1e12,
                         "unit": "T FMA/s", "frac": fma / apply_s / FP32_FMA_PEAK,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def csrc_hash(resident: bool = False) -> str:
    """Hash of the device code the DRAM counters under profiles/ were taken on: the tiled stencil kernels
    (csrc/hv_stencil.cu up to the resident kernels) or, for the resident kernels, the file's device code
    up to the host side, with comments and blank space removed.  Counters apply only while that code is
    unchanged."""
    import re
    text = open(os.path.join(ROOT, "paper_2507_10804_gb300", "csrc", "hv_stencil.cu"), "rb").read()
    mark = b"// ------------------------------------------------------------------ "
    cut = text.find(mark + (b"host side" if resident else b"resident kernels"))
    code = text[:cut] if cut >= 0 else text
    code = re.sub(rb"/\*.*?\*/", b"", code, flags=re.S)
    code = re.sub(rb"//[^\n]*", b"", code)
    code = re.sub(rb"\s+", b" ", code)
    h = hashlib.sha256()
    h.update(code)
    return h.hexdigest()[:16]


def dram_traffic() -> dict:
    """ncu DRAM bytes (read + write) per launch from profiles/dram_traffic.txt.

    Each line: <workload>:<kind> <hash of the kernel sources they were taken on> <bytes> <tile ids of the
    forward, recompute and adjoint kernels>; '#' starts a comment.  Returns {(workload, kind, tile id of that
    kind): (hash, bytes)}, so a kind may have a line for each tile shape the autotuner picks.
    """
    out = {}
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as f:
            for ln in f:
                ln = ln.split("#", 1)[0].split()
                if len(ln) == 4 and ":" in ln[0]:
                    wl, kind = ln[0].split(":", 1)
                    tiles = [int(t) for t in ln[3].split(",")]
                    tid = tiles[{"fwd": 0, "advance": 1, "adj": 2}.get(kind, 0)]
                    out[(wl, kind, tid)] = (ln[1], int(ln[2]))
    except OSError:
        pass
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(w, threads: int, nt_s: int):
    """Time the FP64 oracle's H v on `threads` shots of the workload for nt_s steps;
    returns (Gpt-updates/s, seconds, description)."""
    from oracle import oracle as O
    from paper_2507_10804_gb300 import synth
    ns_s = threads
    idx = np.linspace(0, w.ns - 1, ns_s).round().astype(int)
    P = O.Problem(nz=w.nz, nx=w.nx, nb=w.nb, h=w.h, nt=nt_s, dt=w.dt, f0=w.f0, t0=w.t0, vmax=w.vmax,
                  src_iz=w.acq.src_iz[idx], src_ix=w.acq.src_ix[idx], rec_iz=w.acq.rec_iz[idx],
                  rec_ix=w.acq.rec_ix[idx], R=w.R, sigma=w.sigma)
    m = w.m.astype(np.float32).astype(np.float64)
    v = w.v.astype(np.float32).astype(np.float64)
    t = time.perf_counter()
    O.hessian_apply(P, m, v, nthreads=threads)
    sec = time.perf_counter() - t
    upd = 3.0 * P.NZ * P.NX * nt_s * ns_s
    desc = (f"oracle H v on {ns_s} of {w.ns} shots x first {nt_s} of {w.nt} steps (full grid), "
            f"{threads} threads; scaled by Gpt-updates to one full H v")
    return upd / sec / 1e9, sec, desc


def oracle_rows(w):
    """The FP64 oracle of each approximation row timed on the host on one vector (the batched
    workload's 64x64 grid; the quadratic model on 256x256), as it stands: microseconds per vector."""
    from oracle import lowrank_oracle as LO
    from oracle import pdo_oracle as DO
    from oracle import psf_oracle as PO
    from oracle import quadratic_oracle as QO
    from oracle import spd_oracle as SO
    rng = np.random.default_rng(3)
    nz, nx = w.nz, w.nx
    v = rng.standard_normal((nz, nx))

    def per_call(f, min_s=0.2):
        f()
        n, t = 0, time.perf_counter()
        while True:
            f()
            n += 1
            if time.perf_counter() - t > min_s:
                return (time.perf_counter() - t) / n * 1e6

    S, B = 12, 2
    R = (B * S - 1) // 2
    na = (nz - 1 - S // 2) // S + 1
    nb = (nx - 1 - S // 2) // S + 1
    P = rng.standard_normal((na * nb, 2 * R + 1, 2 * R + 1))
    cplx = lambda r, a, b: rng.standard_normal((r, a, b)) + 1j * rng.standard_normal((r, a, b))
    a8, b8 = cplx(8, nz, nx), cplx(8, nz, nx)
    a22, b22 = cplx(22, nz, nx), cplx(22, nz, nx)
    V16 = rng.standard_normal((16, nz, nx))
    lam16 = np.linspace(1.0, 0.1, 16)
    q = QO.make(256, 256, 10.0, [40.0 * 0.8 ** j for j in range(10)])
    v2 = rng.standard_normal((256, 256))
    a32, b32 = np.abs(cplx(32, 256, 256)), cplx(32, 256, 256)
    out = {
        "psf_apply_us": per_call(lambda: PO.apply(P, v[None], S, B)),
        "pdo_apply_us": per_call(lambda: DO.lr_apply(a8, b8, v)),
        "psfplus_apply_us": per_call(lambda: DO.lr_apply(a22, b22, v)),
        "lr_apply_us": per_call(lambda: LO.apply_H(V16, lam16, v, w.h, 1.0, 2500.0)),
        "lr_sample_us": per_call(lambda: LO.apply_sample_factor(V16, lam16, v, w.h, 1.0, 2500.0)),
        "quad_hd_apply_256_us": per_call(lambda: QO.apply_Hd(q, v2)),
        "quad_objective_256_us": per_call(lambda: QO.objective(q, v2, v2, 1.0, 2500.0)),
        "spd_apply_256_rank32_us": per_call(lambda: SO.spd_apply(a32, b32, v2)),
        "cores": 1,
        "what": "numpy FP64 oracle, one vector per call, as it stands; random factors of the benchmark's shapes",
    }
    return out


def updates_per_call(w) -> float:
    """Grid-point updates of one call applying H to the workload's k vectors: 3 fields
    (forward, Born, adjoint) for the first vector, 2 more per extra vector sharing u;
    recomputation from snapshots is not counted."""
    return 3.0 * (w.nz + 2 * w.nb) * (w.nx + 2 * w.nb) * w.nt * w.ns * (1 + 2.0 * (w.k - 1) / 3.0)


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = min(os.cpu_count() or 1, 8)
    nt_s = 120
    upds = []
    for _ in range(args.warmup):
        oracle_sample(w, threads, nt_s)
    tot = 0.0
    desc = ""
    for _ in range(args.steps):
        g, sec, desc = oracle_sample(w, threads, nt_s)
        upds.append(g)
        tot += sec
    gups = float(np.mean(upds))
    val = gups * 1e9 / updates_per_call(w) * w.k
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded layered/faulted velocity model; stands in for the paper's Marmousi)",
        "config": workload_config(w), "gpt_updates_per_s": gups * 1e9,
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_2507_10804_gb300.hv import Problem, kernel_launches, menu_info
    from paper_2507_10804_gb300.parallel import max_over_ranks, shard_problem, shard_shots, sharded_hessian_apply

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # one process per GPU: this rank's block of shots (all of them on one GPU)
    P = shard_problem(Problem, w, rank, world, device=dev) if world > 1 else Problem.from_workload(w, device=dev)
    ns_local = len(shard_shots(w.ns, rank, world))

    def hv_step(mm, vv):
        # H v of all shots: on one GPU the whole apply; on N ranks the rank's extended image,
        # summed over ranks in rank order (NCCL all-gather) and folded once
        if world == 1:
            return P.hessian_apply(mm, vv, ckpt=CKPT)
        return sharded_hessian_apply(lambda: P.hessian_apply_partial(mm, vv, ckpt=CKPT), P.fold)

    m = torch.tensor(w.m, dtype=torch.float32, device=dev)
    v = torch.tensor(w.v, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    graphs = True                             # the H v launch sequence replays as one CUDA graph
    if args.tiles:                            # fixed tiles (profiling runs: no tuning launches)
        P.set_tiles(args.tiles)
        tiles = P.tiles()
    else:
        tiles = P.autotune(k=w.k)             # fastest tile shape per kernel kind for this grid
    if graphs:
        P.set_graphs(True)
    # the batched workload stores every level on a grid whose field fits in shared memory: H v runs
    # the resident kernels (one persistent launch each for the forward, Born and adjoint fields)
    resident = args.workload == "batched" and CKPT < 0 and not args.no_resident and P.set_resident(True)

    for _ in range(args.warmup):
        hv_step(m, v)
    torch.cuda.synchronize(dev)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = vis.split(",")[local] if vis else str(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_index) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        n0 = kernel_launches()
        e0.record(st)
        for _ in range(args.steps):
            hv_step(m, v)
        e1.record(st)
        torch.cuda.synchronize(dev)
        n1 = kernel_launches()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    # Per-kernel times: the same steps again with an event pair around every launch
    # (on the launching stream).  Kept out of the headline region: the extra event
    # records cost ~6% of the step time.
    P.set_graphs(False)
    P.profile(True)
    P.profile_read()
    ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0 = kernel_launches()
    ep0.record(st)
    for _ in range(args.steps):
        hv_step(m, v)
    ep1.record(st)
    torch.cuda.synchronize(dev)
    if graphs:
        n1 = n0 + (kernel_launches() - c0)          # a graph replay launches the same kernels
    prof = P.profile_read()
    P.profile(False)
    ms_profiled = ep0.elapsed_time(ep1)
    ms_max = max_over_ranks(ms, device=dev)
    calls_per_s = args.steps / (ms_max / 1e3)      # whole H v calls (all shots) per second
    value = calls_per_s * w.k                      # H v products per second (k per call)

    one_at_a_time = None
    if args.workload == "batched" and rank == 0:
        # the plain path: one vector per call, no graph, default tiles (8 of the 64 vectors)
        Q = Problem.from_workload(w, device=dev)
        vs = [v[j:j + 1].contiguous() for j in range(8)]
        Q.hessian_apply(m, vs[0], ckpt=CKPT)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for x in vs:
            Q.hessian_apply(m, x, ckpt=CKPT)
        torch.cuda.synchronize(dev)
        one_at_a_time = {"value": len(vs) / (time.perf_counter() - t0), "unit": UNIT,
                         "what": "one vector per call, stream launches, default tiles (8 vectors timed)"}
        Q.close()
    psf = psf_measure(P, m, w, dev) if args.workload == "batched" and rank == 0 else None
    pdo = pdo_measure(P, m, w, dev) if args.workload == "batched" and rank == 0 else None
    psfplus = psfplus_measure(P, m, w, dev) if args.workload == "batched" and rank == 0 else None
    lowrank = lr_measure(P, m, w, dev) if args.workload == "batched" and rank == 0 else None
    quad = quad_measure(dev) if args.workload == "batched" and rank == 0 else None
    # serving sample (1 GPU): the request mix of the serving workload, 36 requests with 8, 16 or 32 shots, at 2x
    # the serial capacity, with and without merging, against one request at a time
    serve = None
    if args.workload == "paper" and world == 1 and not args.no_serve and args.nt is None and args.shots is None:
        serve = serve_measure(dev, serve_requests(36, shots=[8, 16, 32]), [2.0], 16, batching=(64, 0))
    # end to end through the public API with host buffers (pinned), copies inside the timed region
    mh = torch.tensor(w.m, dtype=torch.float32).pin_memory()
    vh = torch.tensor(w.v, dtype=torch.float32).pin_memory()
    out_h = torch.empty(v.shape, dtype=torch.float32).pin_memory()
    md, vd = torch.empty_like(m), torch.empty_like(v)
    ke = max(1, args.steps)                        # as many calls as the device-timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(ke):
        md.copy_(mh, non_blocking=True)
        vd.copy_(vh, non_blocking=True)
        Hv = hv_step(md, vd)
        out_h.copy_(Hv, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / ke
    e2e_val = w.k / max_over_ranks(e2e_s, device=dev)

    if rank == 0:
        pk, pk_kind = peaks()
        NZ, NX = w.nz + 2 * w.nb, w.nx + 2 * w.nb
        pts = NZ * NX * ns_local
        # algorithmic bytes per time step of each kernel kind, and the steps each kind ran: one per
        # forward+Born and adjoint launch; the recomputation runs fused double steps where it can
        alg = {"fwd": pts * (16 + 16 * w.k), "advance": pts * 16, "adj": pts * (4 + 16 * w.k)}
        from paper_2507_10804_gb300.hv import checkpoint_schedule
        adv_steps = (checkpoint_schedule(w.nt, CKPT)[1] if CKPT > 0 else 0) * args.steps
        kernels = {}
        steps_of = {}
        for kind, (n, tms) in prof.items():
            if n:
                # a resident launch advances all nt steps (the forward kind: forward fields, then Born fields)
                steps_of[kind] = adv_steps if kind == "advance" else (w.nt * args.steps if resident else n)
                kernels[kind] = {"launches_per_step": n / args.steps, "ms_per_step": tms / args.steps,
                                 "avg_launch_us": tms / n * 1e3}
                if kind in alg:
                    kernels[kind]["steps_per_launch"] = steps_of[kind] / n
                    kernels[kind]["algorithmic_GBps"] = alg[kind] * steps_of[kind] / (tms / 1e3) / 1e9
        dom = max(alg, key=lambda k: prof[k][1])
        n_dom, t_dom = prof[dom]
        achieved = alg[dom] * steps_of.get(dom, n_dom) / (t_dom / 1e3) / 1e9
        traffic = None
        # counters recorded for this workload, these kernel sources and these tiles (full-size launches)
        tid = 0 if resident else list(tiles)[{"fwd": 0, "advance": 1, "adj": 2}[dom]]   # the kernel's own tiles
        ent = dram_traffic().get((args.workload + ("-resident" if resident else ""), dom, tid))
        # (taken on all 32 shots: a rank's shot block has other per-launch bytes)
        if ent and ent[0] == csrc_hash(resident) and args.nt is None and args.shots is None and world == 1:
            traffic = ent[1]
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                "algorithmic_bytes_per_launch": alg[dom] * steps_of.get(dom, n_dom) / max(n_dom, 1),
                "peak_source": pk_kind}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            threads = min(os.cpu_count() or 1, 8)
            g, sec, desc = oracle_sample(w, threads, 120)
            cpu = {"value": g * 1e9 / updates_per_call(w) * w.k, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": desc, "seconds": sec, "gpt_updates_per_s": g * 1e9}
            if args.workload == "batched":
                cpu["rows"] = oracle_rows(w)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded layered/faulted velocity model; stands in for the paper's Marmousi)",
            "config": workload_config(w),
            "gpt_updates_per_s": calls_per_s * updates_per_call(w),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT,
                    "h2d_bytes_per_step": int(mh.numel() * 4 + vh.numel() * 4),
                    "d2h_bytes_per_step": int(out_h.numel() * 4)},
            "gpu_launches": int(n1 - n0),
            "profiled_pass": {"ms_per_step": ms_profiled / args.steps,
                              "what": "kernels and roofline: the same steps rerun with CUDA events around every launch"},
            "clocks": clk.summary(),
            "kernels": kernels,
        }
        line["config"]["tiles"] = list(tiles)
        line["config"]["tile_configs"] = [menu_info(c) for c in tiles]
        line["config"]["launch"] = ("H v launch sequence replayed as a CUDA graph; " +
                                    ("shared-memory-resident kernels: one launch each for the forward fields "
                                     "of all shots, the Born fields and the adjoint fields of all (shot, vector) "
                                     "pairs, fields held on chip for all steps" if resident else
                                     "stencil steps with programmatic dependent launch"))
        line["config"]["resident"] = bool(resident)
        line["config"]["parallelism"] = (f"shots split over {world} ranks ({ns_local} on rank 0); FP64 extended "
                                         "images gathered over NCCL, summed in rank order, folded once"
                                         if world > 1 else "1 GPU, all shots")
        if one_at_a_time is not None:
            line["one_at_a_time"] = one_at_a_time
        if serve is not None:
            on = [r for r in serve["runs"] if r["batching_max_vectors"] > 0][0]
            off = [r for r in serve["runs"] if r["batching_max_vectors"] == 0][0]
            line["serve"] = {
                "what": "36 requests (H v 35% / gradient 35% / misfit 15% / PSF-approximation apply 15%) on "
                        "{128x128, 256x256, 384x1152} x {8, 16, 32} shots, Poisson arrivals at 2x the serial "
                        "capacity, 16 streams, 150 GB pool; latency from submission to completion",
                "p50_ms": on["p50_ms"], "p99_ms": on["p99_ms"], "throughput_req_s": on["throughput_req_s"],
                "hv_per_s": on["hv_per_s"], "merged_requests": on["merged_requests"],
                "no_merging": {"p50_ms": off["p50_ms"], "p99_ms": off["p99_ms"],
                               "throughput_req_s": off["throughput_req_s"], "hv_per_s": off["hv_per_s"]},
                "one_at_a_time": {"throughput_req_s": serve["serial_req_s"], "hv_per_s": serve["serial_hv_per_s"]},
                "by_kind": on["by_kind"]}
        if psf is not None:
            line["psf_approximation"] = psf
        if pdo is not None:
            line["pdo_approximation"] = pdo
        if psfplus is not None:
            line["psfplus_approximation"] = psfplus
        if lowrank is not None:
            line["lowrank_approximation"] = lowrank
        if quad is not None:
            line["quadratic_model"] = quad
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def misfits_measure(dev, models=64, steps=5, warm=3, nz=128, nx=128, ns=8, nt=1000, tiles=None):
    """Misfits of `models` proposals on the gpCN chains' problem (128x128 at 10 m + 20-cell sponge, 8 shots,
    1000 steps): one forward sweep of all models (hv_misfit_models, CUDA events around `steps` sweeps), the forward
    kernel's time per step with its algorithmic bytes (12 per shot-point plus one coefficient field per model),
    the same misfits one call at a time, and the misfit engine with a new model joining whenever a slot frees."""
    import torch

    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300.hv import MisfitEngine, Problem

    h = 10.0
    m0 = synth.gradient_grf_model(31, nz, nx, h)
    vmax = float(m0.max())
    acq = synth.surface_acquisition(nx, ns, nx // 3)
    w = synth.Workload(name="chains", nz=nz, nx=nx, nb=20, h=h, nt=nt, dt=synth.cfl_dt(h, vmax), f0=10.0, t0=0.15,
                       vmax=vmax, acq=acq, m=m0, v=np.zeros((1, nz, nx)))
    P = Problem.from_workload(w, device=dev)
    default_tiles = list(P.tiles())
    if tiles:
        P.set_tiles(tiles)
    else:
        P.autotune(1)                           # tile shapes timed on this grid (cached per grid and shot count)
    z = synth.smoothed_normal_vectors(37, models, nz, nx, 4.0)
    z /= np.abs(z).max(axis=(1, 2), keepdims=True)
    ms = torch.tensor(np.minimum(m0[None] * (1.0 + 0.03 * z), vmax), dtype=torch.float32, device=dev)
    dobs = P.fwd_model(torch.tensor(m0, dtype=torch.float32, device=dev) * 1.02)
    st = torch.cuda.current_stream(dev)
    for _ in range(warm):
        P.misfit_models(ms, dobs)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        P.misfit_models(ms, dobs)
    e1.record(st)
    torch.cuda.synchronize(dev)
    sweep_ms = e0.elapsed_time(e1) / steps
    P.profile(True)
    P.profile_read()
    P.misfit_models(ms, dobs)
    torch.cuda.synchronize(dev)
    prof = P.profile_read()
    P.profile(False)
    n_fwd, t_fwd = prof["fwd"]
    step_us = t_fwd / max(n_fwd, 1) * 1e3
    pts = (nz + 2 * 20) * (nx + 2 * 20)
    alg = models * pts * (12.0 * ns + 4.0)
    pk, src = peaks()
    for _ in range(2):
        P.misfit(ms[0], dobs)
    torch.cuda.synchronize(dev)
    e0.record(st)
    for i in range(8):
        P.misfit(ms[i], dobs)
    e1.record(st)
    torch.cuda.synchronize(dev)
    one_ms = e0.elapsed_time(e1) / 8
    # the engine: every slot refilled with the next model as soon as it is done (host-driven ticks)
    ent = dram_traffic().get(("misfits", "advance", P.tiles()[1]))
    traffic = ent[1] if ent and ent[0] == csrc_hash() else None     # ncu bytes of this kernel source and tile
    E = MisfitEngine(P, models)
    done, joined, t0 = 0, 0, None
    target = 4 * models
    while done < target:
        while joined < target and E.active < models:
            E.join(ms[joined % models], dobs)
            joined += 1
        fin = E.tick()
        if fin and t0 is None:
            torch.cuda.synchronize(dev)
            t0, base = time.perf_counter(), done + len(fin)
        done += len(fin)
    done_host = done
    torch.cuda.synchronize(dev)
    eng_s = time.perf_counter() - t0
    E.close()
    # the engine's device-resident loop: every slot refilled from another stream as soon as it is reported done
    E = MisfitEngine(P, models)
    loop_st, post_st = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    posted, done, t0 = 0, 0, None
    while posted < models:
        E.post(ms[posted % models], dobs, stream=post_st)
        posted += 1
    E.serve(loop_st)
    while done < target:
        fin, running = E.poll()
        if fin and t0 is None:
            t0, base_l = time.perf_counter(), done + len(fin)
        done += len(fin)
        for _ in fin:
            if posted < target:
                E.post(ms[posted % models], dobs, stream=post_st)
                posted += 1
        if not running and done < target:
            E.serve(loop_st)
        time.sleep(2e-5)
    loop_s = time.perf_counter() - t0
    E.close()
    return {"problem": f"{nz}x{nx} + 20 sponge, {ns} shots, {nt} steps", "models": models, "tiles": list(P.tiles()),
            "untuned_tiles": default_tiles,
            "sweep_ms": sweep_ms, "misfits_per_s": models / sweep_ms * 1e3,
            "step_kernel_us": step_us, "algorithmic_bytes_per_step": alg,
            "achieved_GBps": alg / step_us * 1e-3, "frac": alg / step_us * 1e-3 / pk["hbm_gbs"], "traffic": traffic,
            "peak_GBps": pk["hbm_gbs"], "peak_source": src,
            "one_at_a_time": {"ms": one_ms, "misfits_per_s": 1e3 / one_ms},
            "engine": {"misfits_per_s": (done_host - base) / eng_s, "completed": done_host - base,
                       "what": "host-driven ticks from Python; a new model joins whenever a slot frees"},
            "device_loop": {"misfits_per_s": (done - base_l) / loop_s, "completed": done - base_l,
                            "what": "the engine's device-resident loop; a new model is posted whenever a slot "
                                    "is reported done"},
            "what": "CUDA events around the sweeps; kernel time per step from per-launch events in a separate sweep"}


def serve_requests(n, seed=20250719, shots=None):
    """The request stream of the serving workload: clients 0-63 are MCMC chains,
    64-67 FWI runs; each request draws its kind (H v 35%, gradient 35%, misfit
    15%, apply of the grid's PSF Hessian approximation 15%), its grid from
    {128x128, 256x256, 384x1152} (steps 1000/1500/3000) and its shot count from
    U{4..32} (or uniformly from the list `shots`)."""
    from paper_2507_10804_gb300 import synth
    u = synth.uniform(seed, 4 * n)
    grids = [(128, 128, 1000), (256, 256, 1500), (384, 1152, 3000)]
    out = []
    for i in range(n):
        x = u[4 * i]
        kind = "hv" if x < 0.35 else ("grad" if x < 0.70 else ("misfit" if x < 0.85 else "approx"))
        g = grids[min(int(u[4 * i + 1] * 3), 2)]
        if shots:
            ns = shots[min(int(u[4 * i + 2] * len(shots)), len(shots) - 1)]
        else:
            ns = 4 + min(int(u[4 * i + 2] * 29), 28)
        client = min(int(u[4 * i + 3] * 68), 67)
        out.append({"kind": kind, "grid": g, "ns": ns, "client": client})
    return out


def serve_measure(dev, reqs, rates, concurrency, batching=(64,), seed=7):
    """Serial (one request at a time) and concurrent serving of `reqs` with Poisson arrivals at the
    given fractions of the serial capacity, for each server batching limit (vectors per merged call;
    0: no merging); every request on a grid uses that grid's model (so requests on one problem merge).
    Returns {"serial_req_s", "serial_hv_per_s", "runs": [...]}; latencies from the server's own clock."""
    import torch

    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300.hv import Problem
    from paper_2507_10804_gb300.serve import Server

    n = len(reqs)
    problems, models, data = {}, {}, {}
    for r in reqs:
        nz, nx, nt = r["grid"]
        key = (nz, nx, r["ns"])
        if key not in problems:
            h = 10.0 if nx < 1000 else 8.0
            nb = 20 if nx < 1000 else 40
            if (nz, nx) not in models:
                m = synth.gradient_grf_model(nz * 7 + nx, nz, nx, h) if nx < 1000 else \
                    synth.layered_faulted_model(2025, nz, nx, h)[1]
                models[(nz, nx)] = (m, torch.tensor(m, dtype=torch.float32, device=dev),
                                    torch.tensor(synth.smoothed_normal_vectors(nz + nx, 1, nz, nx), dtype=torch.float32,
                                                 device=dev))
            m = models[(nz, nx)][0]
            vmax = float(m.max())
            acq = synth.surface_acquisition(nx, r["ns"], nx // 3)
            w = synth.Workload(name="serve", nz=nz, nx=nx, nb=nb, h=h, nt=nt, dt=synth.cfl_dt(h, vmax), f0=10.0,
                               t0=0.15, vmax=vmax, acq=acq, m=m, v=np.zeros((1, nz, nx)))
            problems[key] = Problem.from_workload(w, device=dev)
            data[key] = problems[key].fwd_model(models[(nz, nx)][1] * 1.02)
    ckpt = 30
    # one PSF approximation per grid (12-cell lattice, 4 batches), built at the grid's
    # model with the first acquisition drawn on it; approximate-apply requests use it
    approx = {}
    for r in reqs:
        nz, nx, nt = r["grid"]
        if r["kind"] == "approx" and (nz, nx) not in approx:
            approx[(nz, nx)] = problems[(nz, nx, r["ns"])].approx_build_psf(models[(nz, nx)][1], 12, 4, ckpt=ckpt)
    torch.cuda.synchronize()

    def submit(S, r):
        nz, nx, nt = r["grid"]
        P = problems[(nz, nx, r["ns"])]
        _, m, v = models[(nz, nx)]
        d = data[(nz, nx, r["ns"])]
        if r["kind"] == "hv":
            return S.submit_hv(P, m, v, ckpt=ckpt)[0]
        if r["kind"] == "grad":
            return S.submit_grad(P, m, d, ckpt=ckpt)[0]
        if r["kind"] == "approx":
            return S.submit_approx(approx[(nz, nx)], v)[0]
        return S.submit_misfit(P, m, d)[0]

    budget = 150 << 30
    # serial: one request at a time through the same server (the one-request-at-a-time GPU path)
    S = Server(hbm_budget=budget, max_concurrent=1, device=dev)
    S.set_batching(0)
    for r in reqs[:3]:
        S.wait(submit(S, r))
    t0 = time.perf_counter()
    for r in reqs:
        assert S.wait(submit(S, r)) == 0
    t_serial = time.perf_counter() - t0
    S.close()
    serial_rate = n / t_serial
    n_hv = sum(r["kind"] == "hv" for r in reqs)
    kinds = np.array([r["kind"] for r in reqs])
    runs = []
    S = Server(hbm_budget=budget, max_concurrent=concurrency, device=dev)
    S.set_engine_loop(ENGINE_LOOP)
    for limit in batching:
        S.set_batching(limit)
        rng = np.random.default_rng(seed)
        for frac in rates:
            lam = frac * serial_rate
            arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n))
            ids = []
            t0 = time.perf_counter()
            for a, r in zip(arrivals, reqs):
                dt_ = t0 + a - time.perf_counter()
                if dt_ > 0:
                    time.sleep(dt_)
                ids.append(submit(S, r))
            for i in ids:
                assert S.wait(i) == 0
            infos = [S.info(i) for i in ids]
            lat = np.array([i["t_done"] - i["t_submit"] for i in infos]) * 1e3
            span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
            by_kind = {k: {"p50_ms": float(np.percentile(lat[kinds == k], 50)),
                           "p99_ms": float(np.percentile(lat[kinds == k], 99))}
                       for k in ("hv", "grad", "misfit", "approx") if (kinds == k).any()}
            runs.append({"batching_max_vectors": limit, "rate_frac_of_serial": frac, "offered_req_s": lam,
                         "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                         "throughput_req_s": n / span, "hv_per_s": n_hv / span,
                         "merged_requests": int(sum(i["batch"] > 1 for i in infos)), "by_kind": by_kind})
    S.close()
    for A in approx.values():
        A.close()
    for P in problems.values():
        P.close()
    return {"serial_req_s": serial_rate, "serial_hv_per_s": n_hv / t_serial, "runs": runs}


def serve_chains(dev, concurrency, chains=64, fwi=4, steps=4, fwi_iters=2, beta=0.5):
    """Closed-loop request source: `chains` gpCN chains on a 128x128, 8-shot, 1000-step problem
    and `fwi` FWI-like clients (gradient then H v, repeated) on a 256x256, 16-shot, 1500-step problem,
    all submitting to one server.  A chain step: a sample of the Laplace approximation (low-rank
    approximation with the Matern prior, HV_APPROX_INVSQRT request), the gpCN proposal, the misfit of
    the proposal (request), H~ d = H~_d d (HV_APPROX_H request) + R d, and the FP64 acceptance."""
    import threading

    import torch

    from paper_2507_10804_gb300 import synth
    from paper_2507_10804_gb300._lib import HV_APPROX_H, HV_APPROX_INVSQRT
    from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Posterior, Problem, gpcn_accept, gpcn_propose
    from paper_2507_10804_gb300.serve import Server

    def problem(nz, nx, ns, nt, seed):
        h = 10.0
        m = synth.gradient_grf_model(seed, nz, nx, h)
        vmax = float(m.max())
        acq = synth.surface_acquisition(nx, ns, nx // 3)
        w = synth.Workload(name="serve", nz=nz, nx=nx, nb=20, h=h, nt=nt, dt=synth.cfl_dt(h, vmax), f0=10.0, t0=0.15,
                           vmax=vmax, acq=acq, m=m, v=np.zeros((1, nz, nx)))
        P = Problem.from_workload(w, device=dev)
        mt = torch.tensor(m, dtype=torch.float32, device=dev)
        return P, mt, P.fwd_model(mt * 1.02)

    Pc, mc, dc = problem(128, 128, 8, 1000, 31)
    Pf, mf, df = problem(256, 256, 16, 1500, 32)
    delta, gamma = 1.0, 2500.0
    omega = torch.tensor(synth.normal(33, 24 * 128 * 128).reshape(24, 128, 128), dtype=torch.float32, device=dev)
    LR = Pc.approx_build_lr(mc, delta, gamma, 16, omega, ckpt=30)
    prior = Posterior(128, 128, 10.0, delta, gamma, device=dev)
    vf = torch.tensor(synth.smoothed_normal_vectors(34, 1, 256, 256), dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    S = Server(hbm_budget=150 << 30, max_concurrent=concurrency, device=dev)
    S.set_engine_loop(ENGINE_LOOP)
    rids = {"sample": [], "misfit": [], "hd": [], "grad": [], "hv": []}
    lock = threading.Lock()
    accepted = []
    errors = []

    def note(kind, rid):
        with lock:
            rids[kind].append(rid)

    def chain(c):
        try:
            st = torch.cuda.Stream(device=dev)
            gen = torch.Generator(device=dev).manual_seed(100 + c)
            with torch.cuda.stream(st):
                m = mc.clone()[None].contiguous()
                delta_cur = torch.zeros(1, dtype=torch.float64, device=dev)
                st.synchronize()
                rid, phi0 = S.submit_misfit(Pc, m[0], dc)        # at m0: no prior term
                assert S.wait(rid) == 0
                note("misfit", rid)
                zero = torch.zeros_like(m)
                gpcn_accept(phi0.reshape(1), m, zero, zero, torch.full((1,), -float("inf"), dtype=torch.float64,
                                                                           device=dev), m, delta_cur)
                acc = 0
                for _ in range(steps):
                    n = torch.randn((1, 128, 128), device=dev, generator=gen)
                    st.synchronize()
                    rid, zeta = S.submit_approx(LR, n, HV_APPROX_INVSQRT)
                    assert S.wait(rid) == 0
                    note("sample", rid)
                    m_new, d_new = gpcn_propose(m, mc, zeta, beta)
                    st.synchronize()
                    rid, phi = S.submit_misfit(Pc, m_new[0], dc)
                    rid2, hd = S.submit_approx(LR, d_new, HV_APPROX_H)
                    assert S.wait(rid) == 0 and S.wait(rid2) == 0
                    note("misfit", rid)
                    note("hd", rid2)
                    Rd = prior.apply(d_new)
                    Hd = hd + Rd
                    # Phi = data misfit + prior term 1/2 (m' - m_pr)^T R (m' - m_pr); here m_map = m_pr = m0
                    phi_full = phi.reshape(1) + 0.5 * (d_new.double() * Rd.double()).sum()
                    log_u = torch.log(torch.rand(1, dtype=torch.float64, device=dev, generator=gen))
                    acc += int(gpcn_accept(phi_full, m_new, d_new, Hd, log_u, m, delta_cur).item())
                with lock:
                    accepted.append(acc)
        except Exception as ex:       # reported below
            errors.append(repr(ex))

    def fwi_client(i):
        try:
            for _ in range(fwi_iters):
                rid, _, _ = S.submit_grad(Pf, mf, df, ckpt=30)
                assert S.wait(rid) == 0
                note("grad", rid)
                rid, _ = S.submit_hv(Pf, mf, vf, ckpt=30)
                assert S.wait(rid) == 0
                note("hv", rid)
        except Exception as ex:
            errors.append(repr(ex))

    threads = [threading.Thread(target=chain, args=(c,)) for c in range(chains)]
    threads += [threading.Thread(target=fwi_client, args=(i,)) for i in range(fwi)]
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    span = time.perf_counter() - t0
    if errors:
        raise RuntimeError("chain clients failed: " + errors[0])
    out = {"chains": chains, "fwi_clients": fwi, "chain_steps": chains * steps, "span_s": span,
           "chain_steps_per_s": chains * steps / span, "acceptance": sum(accepted) / (chains * steps),
           "requests": sum(len(v) for v in rids.values()), "requests_per_s": sum(len(v) for v in rids.values()) / span}
    for kind, ids in rids.items():
        lat = np.array([(lambda i: i["t_done"] - i["t_submit"])(S.info(r)) for r in ids]) * 1e3
        if len(lat):
            out[kind] = {"n": len(lat), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                         "mean_batch": float(np.mean([S.info(r)["batch"] for r in ids]))}
    S.close()
    for x in (LR, prior):
        x.close()
    out["what"] = ("closed loop: each chain waits for its requests; sample = LR sampling factor, hd = LR H~_d apply "
                   "(both approximation requests), misfit on the 128x128 problem; FWI clients: gradient and H v on "
                   "256x256")
    return out


def run_serve(args):
    """Serving workload: Poisson arrivals at fractions of the measured serial
    capacity, memory-budgeted admission into a 150 GB pool, with and without
    merging queued requests on one problem and model."""
    import torch

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = args.requests
    reqs = serve_requests(n)
    res = serve_measure(dev, reqs, args.rates, args.concurrency, batching=(64, 0))
    best = max(res["runs"], key=lambda x: x["throughput_req_s"])
    line = {
        "metric": METRIC, "value": best["hv_per_s"], "unit": UNIT, "n_gpus": 1, "steps": n, "warmup": 3,
        "ms_per_step": 1e3 / best["throughput_req_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic request stream (seeded models; stands in for the paper's MCMC and FWI clients)",
        "config": {"workload": "serving: 64 MCMC chains + 4 FWI runs, Poisson arrivals, H v 35% / gradient 35% / "
                               "misfit 15% / PSF-approximation apply 15%, grids {128x128, 256x256, 384x1152} x "
                               "U{4..32} shots, 150 GB pool",
                   "requests": n, "concurrency": args.concurrency, "snapshots_per_shot": 30},
        "serve": res,
    }
    # the first run in a process carries one-time costs (module loading, plans, graph capture) into its latencies
    line["serve"]["gpcn_request_source_first_run"] = serve_chains(dev, args.concurrency)
    line["serve"]["gpcn_request_source"] = serve_chains(dev, args.concurrency)
    print(json.dumps(line))


def main():
    global CKPT, ENGINE_LOOP
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=int(os.environ.get("WORLD_SIZE", "1")))
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nt", type=int, default=None, help="override the step count (profiling runs)")
    ap.add_argument("--shots", type=int, default=None, help="override the shot count (profiling runs)")
    ap.add_argument("--ckpt", type=int, default=None, help="snapshots per shot (profiling runs)")
    ap.add_argument("--requests", type=int, default=60, help="serving workload: requests per rate")
    ap.add_argument("--concurrency", type=int, default=16, help="serving workload: concurrent requests")
    ap.add_argument("--rates", type=float, nargs="+", default=[0.25, 0.5, 0.8, 1.0, 2.0],
                    help="serving workload: arrival rates as fractions of the serial capacity")
    ap.add_argument("--workload", choices=["paper", "batched", "serve", "quadratic", "misfits"], default="paper",
                    help="paper: 384x1152, 32 shots, 3000 steps, 1 vector (default); batched: the 64x64 model "
                         "with 64 vectors x 32 shots x 600 steps, every level stored, CUDA graph; quadratic: "
                         "the quadratic test model's approximation, posterior and gpCN measurements alone; "
                         "misfits: 64 gpCN proposals' misfits in one sweep and through the misfit engine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--engine-loop", action="store_true",
                    help="serving: misfit lanes served by the engine's device-resident loop instead of host ticks")
    ap.add_argument("--no-serve", action="store_true", help="paper workload: skip the serving sample")
    ap.add_argument("--no-resident", action="store_true", help="batched workload: the tiled per-step kernels")
    ap.add_argument("--tiles", type=int, nargs=3, default=None, metavar=("FWD", "ADVANCE", "ADJ"),
                    help="tile configurations instead of autotuning (profiling runs)")
    args = ap.parse_args()
    ENGINE_LOOP = args.engine_loop
    from paper_2507_10804_gb300 import synth
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "quadratic":
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        res = quad_measure(dev, steps=args.steps, warm=args.warmup)
        print(json.dumps({"metric": "gpCN chain steps/s on the quadratic test model (section 4.1)",
                          "value": res["gpcn_steps_per_s"], "unit": "chain steps/s", "n_gpus": 1,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["gpcn_ms_per_step"],
                          "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": f"quadratic model {res['grid'][0]}x{res['grid'][1]}, "
                                                 f"{res['chains']} chains"}, "quadratic_model": res}))
        return
    if args.workload == "misfits":
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        res = misfits_measure(dev, steps=args.steps, warm=args.warmup, tiles=args.tiles)
        print(json.dumps({"metric": "misfits/s of 64 gpCN proposals (section 2.3)", "value": res["misfits_per_s"],
                          "unit": "misfits/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": res["sweep_ms"], "higher_is_better": True, "dtype": "f32",
                          "data": "synthetic", "config": {"workload": f"misfits of {res['models']} models, "
                                                                      f"{res['problem']}"},
                          "roofline": {"bound": "hbm", "kernel": "forward step (all models)",
                                       "achieved": res["achieved_GBps"], "peak": res["peak_GBps"], "unit": "GB/s",
                                       "frac": res["frac"], "traffic": res["traffic"],
                                       "peak_source": res["peak_source"]},
                          "misfits": res}))
        return
    if args.workload == "batched":
        CKPT = args.ckpt if args.ckpt is not None else -1
        w = synth.workload(3, nt=args.nt, ns=args.shots)
    else:
        CKPT = args.ckpt if args.ckpt is not None else 30
        w = synth.workload(2, nt=args.nt, ns=args.shots)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
