"""Benchmark of the UH matrix-vector product on one GB300 (or N independent replicas).

Workload: the unit-sphere Helmholtz collocation operator, N = 32768 Fibonacci points, k = 16,
leaf 64, eta = 1, eps = 1e-6 (ACA 1e-8), stored complex64 with FP32 accumulation, one right-hand
side (complex normal, seed 0). The operator is built on the GPU by the library's builder
(uh_build.h, the host builder is timed beside it), uploaded once, and then timed:

  value     UH matvecs/s, x and y resident on the GPU, matvecs back to back between two CUDA
            events on the launching stream for at least one second (the packed operator, about
            720 MB, is several times the L2 and each matvec streams all of it); the same with an
            L2 flush before every matvec is reported beside it;
  e2e       the same through host buffers: pinned x copied in, matvec, y copied out;
  roofline  algorithmic bytes of one UH matvec (stored operator + vectors, Section 4.4) per
            event-timed matvec, against the measured HBM copy bandwidth;
  extra     the plain H-matrix matvec (Algorithm 5) on the same GPU, the complex128 UH matvec
            against the measured FP64 rate, storage of both forms; the multi-RHS product
            uh_matmat on the tensor cores (TF32 and BF16x3, 32 and 64 right-hand sides) and on
            the CUDA cores (4 per pass); the N = 131072 ellipsoid's 64-RHS product; 32 operators
            of the batched workload in one launch (default and tuned packing); the factored
            coefficient storage; the construction times;
  cpu_baseline  the FP64 oracle's UH matvec on the same operator, timed on one host core in a
            spawned child process, also giving the relative error of the GPU result.

  serving   GMRES(30) solves from a pool of 8 resident operators of the serving distribution (N up
            to 65536) with Poisson arrivals at 50 to 2000 per second: solve latency p50 / p99,
            solves per second, and the share of Arnoldi steps whose product ran in a shared pass.

`--serve` runs the serving sweep alone (pool of 64 operators, N up to 65536, six arrival rates by
default); `--batched` times 256 independent operators in one launch against one launch each.
`--impl reference` times that oracle matvec alone (the reference arm), on the operator made by
the host builder. Under torchrun every
rank runs its own replica (the product has no exchange step to shard), rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "UH matvec/s & HBM GB/s vs H-matvec, same GB300, relerr≤5e-6; solve p50/p99"
UNIT = "matvec/s"


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi sampled every 100 ms while running (SM clock, max clock, throttle reasons)."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- oracle child


def _oracle_child(npz_path: str, out_path: str, seconds: float, min_reps: int, warmup: int = 1):
    """Runs in a fresh process with one BLAS thread: the oracle's UH matvec on the operator in
    npz_path, first on x (result saved for the error check) and `warmup - 1` more times untimed,
    then repeated until both ~seconds and min_reps are reached."""
    import types
    from oracle import uh_oracle as O
    z = {f[:-4]: np.load(os.path.join(npz_path, f), mmap_mode="r")
         for f in os.listdir(npz_path) if f.endswith(".npy")}
    n = int(z["n"])
    begin, size, perm = z["cl_begin"], z["cl_size"], z["perm"]
    tree = types.SimpleNamespace(n=n, perm=perm, begin=begin.tolist(), size=size.tolist())

    def blocks(rank, off, data, clusters):
        return {int(c): data[off[c]:off[c] + size[c] * rank[c]].reshape(rank[c], size[c]).T
                for c in clusters}
    rows = sorted(set(z["adm_row"].tolist()))
    cols = sorted(set(z["adm_col"].tolist()))
    U = blocks(z["row_rank"], z["row_off"], z["U_data"], rows)
    V = blocks(z["col_rank"], z["col_off"], z["V_data"], cols)
    S = {}
    for t, s, o in zip(z["adm_row"], z["adm_col"], z["S_off"]):
        lt, ls = int(z["row_rank"][t]), int(z["col_rank"][s])
        S[(int(t), int(s))] = z["S_data"][o:o + lt * ls].reshape(ls, lt).T
    near = {}
    for t, s, o in zip(z["dense_row"], z["dense_col"], z["D_off"]):
        m, k = int(size[t]), int(size[s])
        near[(int(t), int(s))] = z["D_data"][o:o + m * k].reshape(k, m).T
    adm = sorted(S)
    uh = O.UHMatrix(tree, adm, sorted(near), U, V, S, near, {}, {})
    x = z["x"]
    y = O.uh_matvec(uh, x)
    for _ in range(warmup - 1):
        O.uh_matvec(uh, x)
    reps, t0 = 1, time.perf_counter()
    t_first = None
    while True:
        O.uh_matvec(uh, x)
        reps_done = reps
        reps += 1
        el = time.perf_counter() - t0
        if t_first is None:
            t_first = el
        if el >= seconds and reps_done >= min_reps:
            break
    np.save(out_path + ".y.npy", y)
    with open(out_path, "w") as f:
        json.dump({"reps": reps_done, "seconds": el}, f)


def dump_operator(model, x: np.ndarray, directory: str) -> None:
    """Write the UH descriptor arrays (and x) as .npy files, straight from the builder's memory."""
    for k, v in model.uh_arrays(copy=False).items():
        if v is not None:  # S_rank is None for dense coefficient matrices
            np.save(os.path.join(directory, k + ".npy"), np.asarray(v))
    np.save(os.path.join(directory, "x.npy"), x)


def run_oracle_sample(directory: str, seconds: float, min_reps: int = 2, warmup: int = 1):
    """Spawn the oracle child on the dumped operator (memory-mapped); returns
    (matvec/s, reps, seconds, y)."""
    out = os.path.join(directory, "res.json")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", directory, out,
                    str(seconds), str(min_reps), str(max(1, warmup))], check=True, env=env, cwd=ROOT)
    r = json.load(open(out))
    y = np.load(out + ".y.npy")
    return r["reps"] / r["seconds"], r["reps"], r["seconds"], y


# ----------------------------------------------------------------------------- GPU arm


def replica_times(ms, e2e_ms, dist, device):
    """Per-step times of this rank -> the slowest rank's (all-reduce MAX over the process group),
    which set the whole job's time; unchanged without a process group."""
    if dist is None:
        return ms, e2e_ms
    import torch
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0]), float(t[1])


def job_value(world, ms_max):
    """Whole-job products per second: every rank runs its own replica, one product per step."""
    return world * 1e3 / ms_max


def timed_back_to_back(op, x, y, steps, torch):
    """Mean CUDA-event time (ms) of `steps` matvecs launched back to back on the current stream."""
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(steps):
        op.matvec(x, y)
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


# DRAM bytes (read + write) that ncu counted for one launch of the complex64 stream kernel on the
# N=32768 sphere workload (cold L2), and digests of the code (kernel, packer and program
# construction, comments aside) it was taken on. The figure is reported only while that code is
# unchanged.
NCU_TRAFFIC_BYTES = 717331200
NCU_TRAFFIC_SOURCES = {
    "paper_2405_15573_gb300/csrc/uh_stream.cu": "4028d86a611691b6fa3ea462c2034d13eab53409660ac4238ffa820d42709dbe",
    "paper_2405_15573_gb300/csrc/uh_stream.h": "1e67ea6ae222355a1c22c4d6dc855d67d6c49b5e5e51520698fda7d648c6303d",
    "paper_2405_15573_gb300/csrc/uh_program.cpp": "51c40e8a55be745ce44e8ff4213a5edad1f263293a8784bb45a50033a19dbdca",
    "paper_2405_15573_gb300/csrc/uh_program.h": "d94746040b424e0b03579697ce2690624a5ae7c14a82bce341b2131c19a43527",
    "paper_2405_15573_gb300/csrc/uh_capi.cpp": "ba8249e3eaeb61bec3f1957bb3b0f7e42f092dc6624c95b559ed2b1ba1624d12",
}


def _code_digest(path):
    """sha256 of a C++/CUDA source with its comments and whitespace removed: edits of comments do
    not change the code the counters were taken on."""
    import hashlib
    import re
    with open(path, encoding="utf-8") as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return hashlib.sha256(re.sub(r"\s+", "", src).encode()).hexdigest()


def _traffic():
    for rel, digest in NCU_TRAFFIC_SOURCES.items():
        if _code_digest(os.path.join(ROOT, rel)) != digest:
            return None
    return NCU_TRAFFIC_BYTES


def timed_matvecs(op, x, y, steps, flush, torch):
    """Per-matvec CUDA-event times (ms) with an L2 flush (outside the events) before each."""
    s = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(s)
        op.matvec(x, y)
        b.record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _colmajor_rhs(torch, n, nrhs, seed0=100):
    """n x nrhs column-major complex64 CUDA tensor of seeded complex normal columns."""
    from paper_2405_15573_gb300 import inputs as I
    X = np.stack([I.complex_normal(n, seed0 + j) for j in range(nrhs)], axis=0)
    return torch.from_numpy(X.astype(np.complex64)).to("cuda").T


def matmat_figures(model, n, steps, torch, peak_bf16, sizes=(32, 64)):
    """uh_matmat on the tensor cores (TF32, BF16x3) for 32 and 64 right-hand sides: mean time per
    call (CUDA events, back to back), right-hand-side products per second, bytes of the packed
    operator streamed per second, MMA throughput, and the relative error of each column against
    the CUDA-core product of the same operator (complex64 storage, FP32 accumulation)."""
    out = {}
    ref_op = model.uh_op("c64")
    X64 = _colmajor_rhs(torch, n, 64)
    Yref = torch.empty((64, n), dtype=torch.complex64, device="cuda").T
    ref_op.matmat(X64, Yref, mode="simt")
    ref_op.check()
    yref = Yref.cpu().numpy().astype(np.complex128)
    del ref_op
    # TF32 has half the BF16 tensor rate (2.25 vs 1.1 PFLOP/s nominal dense).
    peaks = {"tf32": peak_bf16 * 1.1 / 2.25, "bf16x3": peak_bf16}
    for mode in ("tf32", "bf16x3"):
        op = model.uh_op("c64_" + mode)
        st = op.stats()
        for nrhs in sizes:
            X = X64[:, :nrhs]
            Y = torch.empty((nrhs, n), dtype=torch.complex64, device="cuda").T
            for _ in range(3):
                op.matmat(X, Y, mode=mode)
            ms = timed_back_to_back(_MatmatStep(op, X, Y, mode), None, None, steps, torch)
            op.check()
            y = Y.cpu().numpy().astype(np.complex128)
            err = max(float(np.linalg.norm(y[:, j] - yref[:, j]) / np.linalg.norm(yref[:, j]))
                      for j in range(nrhs))
            # every MMA of one pass: 2 M N K (3 products in BF16x3), M = 128; a pass of at most 32
            # right-hand sides issues the same MMAs with M = 64
            flops = st["panel_mma_flops"] // (2 if nrhs <= 32 else 1)
            tf = flops / (ms * 1e-3) / 1e12
            out[f"{mode}_R{nrhs}"] = {
                "ms": ms, "rhs_matvec_per_s": nrhs * 1e3 / ms,
                "operator_GBps": st["panel_bytes"] / (ms * 1e-3) / 1e9,
                "mma_m": 64 if nrhs <= 32 else 128,
                "tensor_tflops": tf, "tensor_peak_tflops": peaks[mode], "tensor_frac": tf / peaks[mode],
                "max_col_relerr_vs_simt": err}
        del op
    # the CUDA-core multi-RHS product: 4 right-hand sides per pass (an op of one CTA per SM)
    # against one product per column
    from paper_2405_15573_gb300 import uh as U
    op = model.uh_op("c64", U.PackParams(0, 0, 0, 0, 1))
    X4 = X64[:, :4]
    Y4 = torch.empty((4, n), dtype=torch.complex64, device="cuda").T
    for _ in range(3):
        op.matmat(X4, Y4, mode="simt")
    ms_cols = timed_back_to_back(_MatmatStep(op, X4, Y4, "simt"), None, None, steps, torch)
    yc = Y4.clone()
    op.reserve(4)
    for _ in range(3):
        op.matmat(X4, Y4, mode="simt")
    ms_r4 = timed_back_to_back(_MatmatStep(op, X4, Y4, "simt"), None, None, steps, torch)
    op.check()
    y = Y4.cpu().numpy().astype(np.complex128)
    out["simt_R4"] = {"ms": ms_r4, "ms_by_columns": ms_cols, "speedup": ms_cols / ms_r4,
                      "rhs_matvec_per_s": 4e3 / ms_r4, "bitwise_equal_to_columns": bool(torch.equal(yc, Y4)),
                      "max_col_relerr_vs_simt": max(float(np.linalg.norm(y[:, j] - yref[:, j]) /
                                                          np.linalg.norm(yref[:, j])) for j in range(4))}
    del op
    return out


class _MatmatStep:
    """Adapter so timed_back_to_back can time one matmat call per step."""

    def __init__(self, op, X, Y, mode):
        self.op, self.X, self.Y, self.mode = op, X, Y, mode

    def matvec(self, _x, _y):
        self.op.matmat(self.X, self.Y, mode=self.mode)


def factored_figures(w, x, y_dense, steps, peak, torch):
    """The same workload with the coefficient matrices stored factored where smaller (Section
    4.2; uhb_params.factored, built on the GPU): bytes and product time beside the dense-S form."""
    from paper_2405_15573_gb300 import uh as U
    t0 = time.time()
    m = U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca, device=True, factored=True)
    build_s = time.time() - t0
    op = m.uh_op("c64")
    m.close()
    st = op.stats()
    y = torch.empty_like(x)
    for _ in range(3):
        op.matvec(x, y)
    torch.cuda.synchronize()
    ms = timed_back_to_back(op, x, y, steps, torch)
    op.check()
    gbs = st["algo_bytes_matvec"] / (ms * 1e-3) / 1e9
    rel = float(torch.linalg.vector_norm(y - y_dense) / torch.linalg.vector_norm(y_dense))
    out = {"matvec_per_s": 1e3 / ms, "ms_mean": ms, "steps": steps, "algo_bytes_per_matvec": st["algo_bytes_matvec"],
           "packed_bytes": st["packed_bytes"], "E_S": st["E_S"], "n_factored": st["n_factored"],
           "n_adm": st["n_adm"], "sum_factored_rank": st["sum_factored_rank"], "n_items": st["n_items"],
           "GBps": gbs, "frac": gbs / peak, "build_s": build_s, "relerr_vs_dense_S": rel,
           "note": "S_b = S_X S_Y^* where k (l_tau + l_sigma) < l_tau l_sigma after recompressing the pair at eps; "
                   "t_b = S_Y^* xhat_sigma as its own phase group before the coupling"}
    op.close()
    return out


def build_models(workloads):
    """Several operators built one after the other on the GPU (uhb_build_helmholtz_gpu)."""
    from paper_2405_15573_gb300 import uh as U
    return [U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca, device=True)
            for w in workloads]


def build_ops(workloads, precision="c64", params=None):
    """Device ops of several operators, each built on the GPU and uploaded (packing parameters
    `params`, None: the defaults), its host model freed before the next one is built."""
    from paper_2405_15573_gb300 import uh as U
    ops = []
    for w in workloads:
        m = U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca, device=True)
        ops.append(m.uh_op(precision, params))
        m.close()
    return ops


def serving_figures(pool_count, n_hi, rates, requests, tol=1e-6, restart=30, true_residual_sample=0, max_active=128,
                    pass_width=2):
    """GMRES(restart) solves served from a pool of resident complex64 UH operators (uh_server):
    per arrival rate, `requests` solves with Poisson arrivals, each on a random operator of the
    pool with a seeded right-hand side. Latency = submission to completion (library clock);
    throughput = completed solves / wall time from the first submission to the last completion.
    Each rate runs max(requests, rate / 5) solves, so that at the high rates the start and the
    drain of the queue take a small part of the wall time. Solves of one operator share their
    Arnoldi products in passes of `pass_width` right-hand sides: 2 on the automatic packing, 4 on
    operators packed for one CTA per SM (the four-wide stages do not fit twice on an SM)."""
    from paper_2405_15573_gb300 import inputs as I
    from paper_2405_15573_gb300 import uh as U
    pool = I.serving_pool(pool_count, n_hi=n_hi)
    t0 = time.time()
    ops = build_ops(pool, params=U.PackParams(0, 0, 0, 0, 1) if pass_width == 4 else None)
    build_s = time.time() - t0
    for o in ops:
        o.reserve(pass_width)
    # up to max_active solves run at once: the more of them share an operator, the more products
    # run in shared passes
    srv = U.Server(max_active=max_active, hbm_budget=48 << 30, queue_capacity=1 << 20)
    for o, w in zip(ops, pool):  # one solve per operator before timing
        srv.wait(srv.submit(o, I.complex_normal(w.n, 7), tol=tol, restart=restart))
    out = {"pool": pool_count, "n_range": [min(w.n for w in pool), max(w.n for w in pool)],
           "operator_bytes_c64": int(sum(o.stats()["algo_bytes_matvec"] for o in ops)),
           "build_s": round(build_s, 1), "tol": tol, "restart": restart, "max_active": max_active,
           "pass_width": pass_width, "rates": {}}
    base_requests = requests
    for lam in rates:
        requests = max(base_requests, int(lam / 5))
        arr = I.poisson_arrivals(lam, requests, seed=int(lam))
        which = np.random.default_rng(int(lam) + 1).integers(0, pool_count, size=requests)
        bs = [I.complex_normal(pool[k].n, 100 + i) for i, k in enumerate(which)]
        tickets = []
        start = time.perf_counter()
        for i in range(requests):
            dt = arr[i] - (time.perf_counter() - start)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(ops[which[i]], bs[i], tol=tol, restart=restart, maxit=20 * restart))
        res = [srv.wait(t, timeout=600) for t in tickets if t is not None]
        wall = time.perf_counter() - start
        lat = np.array([r[1]["latency_s"] for r in res])
        out["rates"][str(int(lam))] = {
            "requests": requests, "refused": sum(t is None for t in tickets),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "solves_per_s": len(res) / wall,
            "iterations_mean": float(np.mean([r[1]["iterations"] for r in res])),
            "paired_step_frac": float(sum(r[1]["paired_steps"] for r in res) /
                                      max(1, sum(r[1]["iterations"] for r in res))),
            "converged_frac": float(np.mean([r[1]["converged"] for r in res])),
            "max_rel_residual": float(max(r[1]["rel_residual"] for r in res))}
    srv.close()
    del ops
    return out


def large_matmat_figures(torch, peak_bf16, steps):
    """The N = 131072 ellipsoid (1, 0.7, 0.4) with 1% radial noise, k = 32, eps 1e-4: uh_matmat
    with 64 right-hand sides in both tensor-core modes, against its CUDA-core product."""
    from paper_2405_15573_gb300 import inputs as I
    from paper_2405_15573_gb300 import uh as U
    w = I.ELLIPSOID_131072_R64
    t0 = time.time()
    model = U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca, device=True)
    build_s = time.time() - t0
    res = matmat_figures(model, w.n, steps, torch, peak_bf16, sizes=(64,))
    st = model.uh_op("c64").stats()
    model.close()
    return {"workload": w.name, "operator_build_s": round(build_s, 1), "operator_build": "GPU (uhb_build_helmholtz_gpu)",
            "algo_bytes_matvec_c64": st["algo_bytes_matvec"], **res}


def batched_figures(count, steps, tune_sample=32):
    """One launch for `count` independent complex64 UH operators (uh_batch) against one launch
    per operator (uh_matvec each), back to back, CUDA events; operator products per second. The
    batch is packed twice: with the default parameters and with the autotuner's choice
    (uh_batch_tune on an evenly spaced sample of `tune_sample` of the operators)."""
    import torch
    from paper_2405_15573_gb300 import inputs as I
    from paper_2405_15573_gb300 import uh as U
    pool = I.batched_pool(count)
    t0 = time.time()
    models = build_models(pool)
    build_s = time.time() - t0
    descs = [m.uh_desc() for m in models]
    t0 = time.time()
    best, tune_best_ms, tune_default_ms = U.UHBatch.tune(descs, "c64", sample=tune_sample, reps=20)
    tune_s = time.time() - t0
    t0 = time.time()
    batch = U.UHBatch(descs, "c64")
    pack_s = time.time() - t0
    tuned = U.UHBatch(descs, "c64", best)
    ops = [m.uh_op("c64") for m in models]
    for m in models:
        m.close()
    off = batch.offsets
    x = torch.from_numpy(np.concatenate([w.x() for w in pool])).to("cuda", torch.complex64)
    y, y2 = torch.empty_like(x), torch.empty_like(x)

    class Seq:
        def matvec(self, _x, _y):
            for k, op in enumerate(ops):
                op.matvec(x[off[k]:off[k + 1]], y2[off[k]:off[k + 1]])
    y3 = torch.empty_like(x)
    for _ in range(3):
        batch.matvec(x, y)
        tuned.matvec(x, y3)
        Seq().matvec(None, None)
    ms_b = timed_back_to_back(batch, x, y, steps, torch)
    ms_t = timed_back_to_back(tuned, x, y3, steps, torch)
    ms_s = timed_back_to_back(Seq(), None, None, max(3, steps // 5), torch)
    batch.check()
    tuned.check()
    tuned_diff = float(torch.linalg.vector_norm(y3 - y) / torch.linalg.vector_norm(y))
    st = batch.stats()
    yb, ys = y.cpu().numpy().astype(np.complex128), y2.cpu().numpy().astype(np.complex128)
    diff = max(float(np.linalg.norm(yb[off[k]:off[k + 1]] - ys[off[k]:off[k + 1]]) /
                     np.linalg.norm(ys[off[k]:off[k + 1]])) for k in range(count))
    peak, _ = _peaks()
    return {"operators": count, "points": int(off[-1]), "build_s": round(build_s, 1), "pack_s": round(pack_s, 1),
            "ms_batched": ms_b, "ms_separate": ms_s, "speedup": ms_s / ms_b,
            "operator_matvecs_per_s": count * 1e3 / ms_b, "operator_matvecs_per_s_separate": count * 1e3 / ms_s,
            "GBps": st["algo_bytes_matvec"] / (ms_b * 1e-3) / 1e9,
            "frac": st["algo_bytes_matvec"] / (ms_b * 1e-3) / 1e9 / peak,
            "algo_bytes": st["algo_bytes_matvec"], "max_rel_diff_vs_separate": diff,
            "tuned": {"params": best.as_dict(), "ms": ms_t, "operator_matvecs_per_s": count * 1e3 / ms_t,
                      "GBps": st["algo_bytes_matvec"] / (ms_t * 1e-3) / 1e9,
                      "frac": st["algo_bytes_matvec"] / (ms_t * 1e-3) / 1e9 / peak,
                      "speedup_vs_default": ms_b / ms_t, "tune_s": round(tune_s, 1),
                      "tune_sample": min(tune_sample, count),
                      "tuner_ms_default_on_sample": tune_default_ms, "tuner_ms_best_on_sample": tune_best_ms,
                      "relative_diff_vs_default": tuned_diff}}


def profile_arm(args):
    """Only one op (uh64, h64 or uh128) of the benchmark workload: build, warm up, run `steps`
    products and print their mean time. For profiler captures of a single kernel."""
    import torch
    from paper_2405_15573_gb300 import inputs as I
    from paper_2405_15573_gb300 import uh as U
    w = I.SPHERE_32768
    model = U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca)
    if args.profile_op.startswith("mm_"):
        mode = args.profile_op[3:]
        op = model.uh_op("c64_" + mode)
        model.close()
        X = _colmajor_rhs(torch, w.n, 64)
        Y = torch.empty((64, w.n), dtype=torch.complex64, device="cuda").T
        run = lambda: op.matmat(X, Y, mode=mode)  # noqa: E731
    elif args.profile_op == "simt_r4":
        # the CUDA-core multi-RHS product: 4 right-hand sides per pass (one CTA per SM)
        op = model.uh_op("c64", U.PackParams(0, 0, 0, 0, 1))
        model.close()
        op.reserve(4)
        X = _colmajor_rhs(torch, w.n, 4)
        Y = torch.empty((4, w.n), dtype=torch.complex64, device="cuda").T
        run = lambda: op.matmat(X, Y, mode="simt")  # noqa: E731
    else:
        prec = "c128" if args.profile_op.endswith("128") else "c64"
        op = model.uh_op(prec) if args.profile_op.startswith("uh") else model.h_op(prec)
        model.close()
        dt = torch.complex128 if prec == "c128" else torch.complex64
        x = torch.from_numpy(w.x()).to("cuda", dt)
        y = torch.empty_like(x)
        run = lambda: op.matvec(x, y)  # noqa: E731
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        run()
    b.record()
    op.check()
    print(json.dumps({"profile_op": args.profile_op, "ms_mean": a.elapsed_time(b) / args.steps,
                      "algo_bytes": op.stats()["algo_bytes_matvec"]}))


def gpu_arm(args):
    import ctypes as C
    import torch
    from paper_2405_15573_gb300 import inputs as I
    from paper_2405_15573_gb300 import uh as U

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = I.SPHERE_32768
    t0 = time.time()
    model = U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca, device=True)
    build_s = time.time() - t0
    build_info = model.info()
    t0 = time.time()
    U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca).close()
    build_host_s = time.time() - t0
    uh64 = model.uh_op("c64")
    h64 = model.h_op("c64")
    uh128 = model.uh_op("c128")
    st = uh64.stats()
    hst = h64.stats()
    x_np = w.x()
    tmpdir = None
    if not args.no_cpu_baseline and rank == 0:
        tmpdir = tempfile.mkdtemp(prefix="uh_bench_")
        dump_operator(model, x_np, tmpdir)
    peak_bf16 = _bf16_peak()
    mm = None if args.no_matmat else matmat_figures(model, w.n, max(10, args.steps // 20), torch, peak_bf16)
    model.close()  # the ops hold their own device copies; free the host arrays
    x = torch.from_numpy(x_np).to("cuda", torch.complex64)
    y = torch.empty_like(x)
    x128 = torch.from_numpy(x_np).to("cuda")
    y128 = torch.empty_like(x128)
    yh = torch.empty_like(x)
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20), dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        uh64.matvec(x, y)
        h64.matvec(x, yh)
        uh128.matvec(x128, y128)
    torch.cuda.synchronize()
    # The timed region runs for at least about one second of wall time: K steps as asked, or more
    # when K steps would take less (estimated from a short untimed run).
    ms_est = timed_back_to_back(uh64, x, y, 20, torch)
    steps_timed = max(args.steps, int(math.ceil(1000.0 / max(ms_est, 1e-3))))

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # The timed region: K UH products back to back. The packed operator (about 720 MB) is several
    # times the L2, and every product streams all of it, so no flush is needed between steps.
    ms_uh = timed_back_to_back(uh64, x, y, steps_timed, torch)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # Secondary figures: H and c128 back to back; the UH product again with a 2x-L2 flush before
    # each step (outside the events).
    ms_h = timed_back_to_back(h64, x, yh, args.steps, torch)
    ms_128 = timed_back_to_back(uh128, x128, y128, max(10, args.steps // 10), torch)
    fp64 = C.c_double(0.0)
    U.check(U.lib.uh_debug_dfma_rate(100000, C.byref(fp64), None), "uh_debug_dfma_rate")
    fp64_tflops = fp64.value
    t_uh_fl = timed_matvecs(uh64, x, y, args.steps, flush, torch)
    # End to end through host buffers: every step copies its x in from pinned host memory, runs
    # the product and copies its y out. Two streams alternate so that a step's copies overlap the
    # neighbouring steps' products; the products themselves are chained by an event in launch
    # order (they share the op's scratch).
    xh = torch.from_numpy(x_np.astype(np.complex64)).pin_memory()
    yhost = [torch.empty_like(xh).pin_memory() for _ in range(2)]
    xd = [torch.empty_like(x) for _ in range(2)]
    yd = [torch.empty_like(y) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = args.steps
    torch.cuda.synchronize()
    e0.record(s)
    for cs in streams:
        cs.wait_event(e0)
    for i in range(e2e_steps):
        k = i & 1
        cs = streams[k]
        with torch.cuda.stream(cs):
            xd[k].copy_(xh, non_blocking=True)
            if i > 0:
                cs.wait_event(done[1 - k])
            uh64.matvec(xd[k], yd[k], stream=cs)
            done[k].record(cs)
            yhost[k].copy_(yd[k], non_blocking=True)
    for cs in streams:
        s.wait_stream(cs)
    e1.record(s)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / e2e_steps
    uh64.check()
    assert np.array_equal(yhost[(e2e_steps - 1) & 1].numpy(), y.cpu().numpy()), "e2e result differs"
    time.sleep(0.2)
    clk = clocks.stop()
    # Configurations beyond the headline, each a documented subset that keeps its size range:
    # the N = 131072 ellipsoid's 64-RHS product (whole), 32 of the 256 batched operators (N
    # log-uniform in [1024, 16384]), and a serving pool of 8 operators with N uniform in
    # [4096, 65536] at the six arrival rates.
    large_mm = None if args.no_matmat or args.quick else large_matmat_figures(torch, peak_bf16, 20)
    factored = factored_figures(w, x, y, max(args.steps, 200), _peaks()[0], torch)
    batched = None if args.quick else batched_figures(32, 20)
    serving = None if args.no_serving else serving_figures(
        8, 65536 if not args.quick else 16384,
        (50, 100, 200, 500, 1000, 2000) if not args.quick else (200, 1000), 150)

    ms_max, t_e2e = replica_times(ms_uh, t_e2e, dist, "cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_kind = _peaks()
    gbs = st["algo_bytes_matvec"] / (ms_uh * 1e-3) / 1e9
    gbs_h = hst["algo_bytes_matvec"] / (ms_h * 1e-3) / 1e9
    gbs_128 = uh128.stats()["algo_bytes_matvec"] / (ms_128 * 1e-3) / 1e9
    traffic = _traffic()
    y_np = y.cpu().numpy().astype(np.complex128)
    y128_np = y128.cpu().numpy()

    cpu = None
    rel_oracle = None
    if tmpdir is not None:
        try:
            rate, reps, secs, y_ref = run_oracle_sample(tmpdir, args.cpu_seconds)
        finally:
            import shutil
            shutil.rmtree(tmpdir, ignore_errors=True)
        rel_oracle = float(np.linalg.norm(y_np - y_ref) / np.linalg.norm(y_ref))
        rel_oracle_128 = float(np.linalg.norm(y128_np - y_ref) / np.linalg.norm(y_ref))
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{reps} full FP64 UH matvecs of the same N=32768 operator "
                         f"(NumPy, one BLAS thread) in {secs:.1f} s",
               "relerr_c64_vs_oracle": rel_oracle, "relerr_c128_vs_oracle": rel_oracle_128}

    out = {
        "metric": METRIC, "value": job_value(world, ms_max), "unit": UNIT, "n_gpus": world,
        "steps": steps_timed, "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "timed_seconds": ms_max * steps_timed / 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic",
        "config": {"workload": workload_name(w),
                   "precision": "complex64 storage, FP32 accumulation",
                   "l2": "inputs larger than L2: the packed operator is "
                         f"{st['packed_bytes'] / 2**20:.0f} MiB, every step streams all of it; no flush",
                   "parallelism": f"replicas x{world}", "operator_build_s": round(build_s, 2),
                   "operator_build": "GPU (uhb_build_helmholtz_gpu, Algorithms 3/4 with ACA on the device)"},
        "e2e": {"value": job_value(world, t_e2e), "unit": UNIT,
                "note": "uh_matvec on two alternating streams; each step's x in and y out overlap neighbouring products",
                "h2d_bytes_per_step": int(x.numel() * 8),
                "d2h_bytes_per_step": int(y.numel() * 8)},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "kernel": ("stream_kernel<KC64Dual> (complex64, two CTAs per SM" if st["pack_ctas_per_sm"] == 2
                                else "stream_kernel<KC64> (complex64, one CTA per SM") +
                               "; one persistent launch per matvec)",
                     "algo_bytes_per_matvec": st["algo_bytes_matvec"],
                     "frac_of_nominal_8000": gbs / 8000.0,
                     "l2_flushed": {"achieved": st["algo_bytes_matvec"] / (statistics.mean(t_uh_fl) * 1e-3) / 1e9,
                                    "frac": st["algo_bytes_matvec"] / (statistics.mean(t_uh_fl) * 1e-3) / 1e9 / peak,
                                    "frac_median": st["algo_bytes_matvec"] / (statistics.median(t_uh_fl) * 1e-3) / 1e9 / peak,
                                    "note": "same kernel, 2x-L2 write before every matvec (outside the events); "
                                            "mean and median over the flushed steps"}},
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": steps_timed * st["n_launches"],
        "uh": {"ms_mean": ms_uh, "GBps": gbs, "relerr_vs_oracle": rel_oracle, "stats": st,
               "flushed": {"ms_mean": statistics.mean(t_uh_fl), "ms_median": statistics.median(t_uh_fl),
                           "ms_min": min(t_uh_fl), "matvec_per_s": 1e3 / statistics.mean(t_uh_fl),
                           "note": "2x-L2 write before every step, outside the events"}},
        "h": {"matvec_per_s": 1e3 / ms_h, "ms_mean": ms_h, "GBps": gbs_h,
              "algo_bytes": hst["algo_bytes_matvec"], "speedup_uh_over_h": ms_h / ms_uh},
        "uh_matmat": mm,
        "serving": serving,
        "uh_c128": {"matvec_per_s": 1e3 / ms_128, "ms_mean": ms_128, "GBps": gbs_128,
                    "bound": "fp64 FMA (8 flops per complex multiply-add of a 16-byte element)",
                    "fp64_tflops": gbs_128 / 16 * 8 / 1e3,
                    "fp64_peak_tflops_measured": fp64_tflops,
                    "fp64_frac": (gbs_128 / 16 * 8 / 1e3) / fp64_tflops,
                    "peak_note": "uh_debug_dfma_rate: 8 independent DFMA chains per thread, 4 CTAs x 256 per SM"},
        "uh_matmat_large": large_mm,
        "uh_factored": dict(factored, ms_dense=ms_uh, bytes_dense=st["algo_bytes_matvec"],
                            speedup_vs_dense=ms_uh / factored["ms_mean"],
                            bytes_ratio=factored["algo_bytes_per_matvec"] / st["algo_bytes_matvec"]),
        "batched": batched,
        "construction": {"gpu_s": build_s, "host_s": build_host_s, "speedup": build_host_s / build_s,
                         "gpu_stages_s": {k: build_info[k] for k in ("seconds_tree", "seconds_aca", "seconds_bases",
                                                                      "seconds_dense")},
                         "host_cores": os.cpu_count(),
                         "note": "same operator from both builders (identical trees; ranks and products agree to rounding)"},
        "storage": {"E_UH": st["E_U"] + st["E_V"] + st["E_S"] + st["E_D"],
                    "E_H": hst["E_U"] + hst["E_V"] + hst["E_D"],
                    "ratio_H_over_UH": (hst["E_U"] + hst["E_V"] + hst["E_D"]) /
                                       (st["E_U"] + st["E_V"] + st["E_S"] + st["E_D"]),
                    "ratio_adm": (hst["E_U"] + hst["E_V"]) / (st["E_U"] + st["E_V"] + st["E_S"])},
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm


def workload_name(w):
    """The benchmark workload, named the same way by both arms."""
    return (f"UH matvec, unit-sphere Helmholtz collocation N={w.n} k={w.wavenumber:g} leaf {w.leaf} "
            f"eta {w.eta:g} eps {w.eps:g}, 1 RHS")


def reference_arm(args):
    """The oracle (FP64 NumPy, one BLAS thread) timed on the benchmark workload: the operator is
    made by the library's host builder (no GPU), written out, and each step is one full oracle UH
    matvec of it in a child process."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2405_15573_gb300 import inputs as I
    from paper_2405_15573_gb300 import uh as U
    w = I.SPHERE_32768
    t0 = time.time()
    model = U.HelmholtzModel(w.points(), w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca)
    build_s = time.time() - t0
    tmpdir = tempfile.mkdtemp(prefix="uh_ref_")
    try:
        dump_operator(model, w.x(), tmpdir)
        model.close()
        rate, reps, secs, _ = run_oracle_sample(tmpdir, 0.0, args.steps, args.warmup)
    finally:
        import shutil
        shutil.rmtree(tmpdir, ignore_errors=True)
    ms = 1e3 * secs / reps
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    out = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world, "steps": reps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_name(w),
                      "precision": "complex128, the FP64 oracle on the host (no GPU work)",
                      "operator_build_s": round(build_s, 1),
                      "operator": "built by the library's host builder (uhb_build_helmholtz, the oracle's "
                                  "algorithm in C++; the oracle's own NumPy construction of N=32768 does not fit "
                                  "the arm's time), then applied by the oracle's FP64 UH product"},
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{reps} full FP64 oracle UH matvecs of the N={w.n} operator "
                                      f"(NumPy, one BLAS thread) in {secs:.1f} s"},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--oracle-child":
        _oracle_child(sys.argv[2], sys.argv[3], float(sys.argv[4]), int(sys.argv[5]), int(sys.argv[6]))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="uh", choices=["uh", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile-op", choices=["uh64", "h64", "uh128", "mm_tf32", "mm_bf16x3", "simt_r4"], default=None)
    ap.add_argument("--no-matmat", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the large matmat and the batch, smaller serving pool")
    ap.add_argument("--serve", action="store_true", help="serving sweep only (pool and rates below)")
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--n-hi", type=int, default=65536)
    ap.add_argument("--rates", default="50,100,200,500,1000,2000")
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--max-active", type=int, default=128, help="serving: solves running at once")
    ap.add_argument("--pass-width", type=int, default=2, choices=[2, 4], help="serving: right-hand sides per shared pass")
    ap.add_argument("--batched", action="store_true", help="batched-operator timing only")
    ap.add_argument("--operators", type=int, default=256)
    args = ap.parse_args()
    if args.batched:
        import torch
        torch.cuda.init()
        print(json.dumps({"batched": batched_figures(args.operators, args.steps or 20)}), flush=True)
        return
    if args.serve:
        import torch
        torch.cuda.init()
        res = serving_figures(args.pool, args.n_hi, [float(v) for v in args.rates.split(",")], args.requests,
                              max_active=args.max_active, pass_width=args.pass_width)
        print(json.dumps({"serving": res}), flush=True)
        return
    if args.profile_op:
        args.steps = 5 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else args.warmup
        profile_arm(args)
        return
    if args.impl == "reference":
        args.steps = 5 if args.steps is None else args.steps
        args.warmup = 1 if args.warmup is None else args.warmup
        reference_arm(args)
        return
    args.steps = 2000 if args.steps is None else args.steps
    args.warmup = 20 if args.warmup is None else max(3, args.warmup)
    gpu_arm(args)


if __name__ == "__main__":
    main()
