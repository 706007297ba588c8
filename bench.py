"""Throughput of full network solves on GB300 (one JSON line on stdout).

A step is one pass of the whole path over one synthetic network already in
device memory: assembly of K from the edge list, the free-dof operator, the
preconditioner set-up (host elements and Q1 values, coarse dofs, Galerkin
matrix and its inverse, star orderings and factors) and PCG to a relative
residual of 1e-8.  The workload is the 3D scalar diffusion network: 40000
fibers of length 0.1 in the unit cube, contacts below 0.004, u = 0 at x < 0.01
and u = 1 at x > 0.99, mesh width H = 1/16, stars at interior mesh nodes.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the library's stream; between steps (outside the events) a 512 MiB buffer
is written to flush the L2.  `value` = K / (sum of step times).  `e2e` repeats
the same steps through the C ABI with host buffers (pinned), the host/device
copies inside the timed region.  Under torchrun every rank solves its own
networks (replicas, no collective) and rank 0 reports the aggregate.

--impl reference times the CPU FP64 oracle on the same workload (the reference
implementation of this build; see the design notes).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2207_07488_gb300 import networks as nw  # noqa: E402

# PCG iterations of the FP64 oracle at rtol 1e-8 on replicate 0 (the CUDA FP64
# path takes the same count; used to extrapolate the bounded CPU samples)
REF_ITERS = {"c2": 152, "c1": 38}

WORKLOADS = {
    # name: (generator, description)
    "c2": (lambda r: nw.config2(replicate=r),
           "3d-diffusion-40000fibers-L0.1-contact0.004-H1/16"),
    "c1": (lambda r: nw.config1(replicate=r), "2d-diffusion-1000fibers-L0.1-H1/8"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--replicates", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, index=0):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        self.index = index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=float(np.median(sm)) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons), samples=len(rows))
        return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes of one launch of the iteration kernels
# ---------------------------------------------------------------------------
def kernel_bytes(op, pc, prec_bytes):
    """Algorithmic bytes of one launch of each iteration kernel: every array the
    kernel must touch, counted once per pass (the star gather counts each star's
    copy of r)."""
    n = op.info.n_free
    nnz = op.info.nnz_ff
    i = pc.info
    ss = i.sum_star
    d = op.dim
    nc = 2 ** d
    vb = prec_bytes                      # factor, coarse inverse and star result bytes
    xb = 8 if prec_bytes == 8 else 4     # local coordinates read by update / combine
    nt = (i.m0 + 127) // 128
    return {
        # values + columns, row pointers (int64), z gathered, p and q read and written
        "spmv": 12 * nnz + 8 * (n + 1) + 8 * n + 32 * n,
        # headers, inverse permutations and window records; r over every star; w written
        "stars": i.star_stream_bytes + 8 * ss + vb * ss,
        # the packed upper tiles of A_0^{-1}; r_c formed from the corner sums
        "coarse": vb * (nt * (nt + 1) // 2) * 128 * 128 + 8 * 8 * i.m0 + 8 * i.m0,
        # x, p, r, q read, x and r written, local coordinates, corner sums written
        "update": 48 * n + xb * d * n + 8 * nc * i.n_elem,
        # local coordinates, star results, r and the old z read, z written
        "combine": xb * d * n + vb * ss + 24 * n,
    }


def run_gb300(args, rank, world, local):
    import torch

    from paper_2207_07488_gb300 import spnet

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gen, desc = WORKLOADS[args.workload]
    probs = [gen(r + 10 * rank) for r in range(args.replicates)]
    prec = spnet.PREC_MIXED if args.precision == "mixed" else spnet.PREC_FP64
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)

    def to_dev(a, dt=None):
        return torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).to(dev)

    dev_inputs = []
    for p in probs:
        net = p.net
        m = net.n_edges
        cap = p.ndof * p.ndof * (net.n_nodes + 2 * m)
        dev_inputs.append(dict(
            edges=to_dev(net.edges, np.int64), coef=to_dev(net.cond), coords=to_dev(net.coords),
            dd=to_dev(p.dirichlet_dofs, np.int64), f=to_dev(p.f), g=to_dev(p.dirichlet_vals),
            rp=torch.zeros(net.n_nodes * p.ndof + 1, dtype=torch.int64, device=dev),
            col=torch.zeros(cap, dtype=torch.int32, device=dev),
            val=torch.zeros(cap, dtype=torch.float64, device=dev)))
    lib = spnet.load()
    import ctypes as C

    sp = C.c_void_p(stream.cuda_stream)

    def one_step(k, host=None):
        p = probs[k % len(probs)]
        d = dev_inputs[k % len(probs)]
        net = p.net
        nnz = C.c_int64(0)
        if host is None:
            spnet._check(lib.spnet_assemble(
                spnet.MODEL_SCALAR, net.n_nodes, net.n_edges, d["edges"].data_ptr(), d["coef"].data_ptr(),
                None, spnet.MEM_DEVICE, sp, d["rp"].data_ptr(), d["col"].data_ptr(), d["val"].data_ptr(),
                d["col"].numel(), C.byref(nnz)))
            op = spnet.Operator(net.dim, p.ndof, d["coords"], d["rp"], d["col"][:nnz.value],
                                d["val"][:nnz.value], d["dd"], net.domain, stream=stream)
            pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=prec)
            x, st = spnet.pcg_solve(op, pc, d["f"], d["g"], rtol=1e-8)
        else:
            h = host[k % len(probs)]
            spnet._check(lib.spnet_assemble(
                spnet.MODEL_SCALAR, net.n_nodes, net.n_edges, h["edges"].ctypes.data, h["coef"].ctypes.data,
                None, spnet.MEM_HOST, sp, h["rp"].ctypes.data, h["col"].ctypes.data, h["val"].ctypes.data,
                h["col"].size, C.byref(nnz)))
            op = spnet.Operator(net.dim, p.ndof, h["coords"], h["rp"], h["col"][:nnz.value],
                                h["val"][:nnz.value], h["dd"], net.domain, stream=stream)
            pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=prec)
            x, st = spnet.pcg_solve(op, pc, h["f"], h["g"], rtol=1e-8)
        info = (op, pc, st[0])
        return info, x

    def timed(n_steps, warm, host=None):
        times, last = [], None
        for k in range(warm + n_steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info, x = one_step(k, host)
            e1.record(stream)
            torch.cuda.synchronize()
            op, pc, st = info
            if not st.converged or st.relres > 1e-8:
                raise RuntimeError(f"solve did not converge: relres={st.relres}")
            if k >= warm:
                times.append(e0.elapsed_time(e1))
            if k == warm + n_steps - 1:
                last = (op.info, pc.info, st, kernel_bytes(op, pc, 8 if prec == spnet.PREC_FP64 else 4))
            pc.close()
            op.close()
        return times, last

    # warm-up, then the timed device-resident steps (CUDA graphs, no instrumentation)
    timed(0, args.warmup)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = spnet.launch_count()
    t_wall0 = time.perf_counter()
    times, last = timed(args.steps, 0)
    t_wall = time.perf_counter() - t_wall0
    l1 = spnet.launch_count()
    clk = clocks.stop()
    torch.cuda.synchronize()
    # a profiled pass over the same steps: every kernel launch timed with CUDA
    # events on its own stream (eager launches, so that each kernel has its events)
    spnet.profile_reset()
    spnet.profile_enable(True)
    ptimes, _ = timed(min(args.steps, 2), 0)
    spnet.profile_enable(False)
    prof = spnet.profile_read()
    torch.cuda.synchronize()
    # e2e: host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host = []
        for p in probs:
            net = p.net
            cap = p.ndof * p.ndof * (net.n_nodes + 2 * net.n_edges)

            def pinned(a, dt):
                t = torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()
                return t.numpy()

            host.append(dict(
                edges=pinned(net.edges, np.int64), coef=pinned(net.cond, np.float64),
                coords=pinned(net.coords, np.float64), dd=pinned(p.dirichlet_dofs, np.int64),
                f=pinned(p.f, np.float64), g=pinned(p.dirichlet_vals, np.float64),
                rp=pinned(np.zeros(net.n_nodes * p.ndof + 1), np.int64),
                col=pinned(np.zeros(cap), np.int32), val=pinned(np.zeros(cap), np.float64)))
        ht, hlast = timed(args.steps, 1, host)
        p = probs[0]
        oi = hlast[0]
        h2d = (p.net.n_edges * 24 + p.net.n_nodes * p.net.dim * 8
               + p.dirichlet_dofs.size * 8 + p.n_dof * 8 + p.dirichlet_vals.size * 8)
        # the assembled CSR goes down to the host and back up to the operator
        nnz_k = (p.net.n_nodes + 2 * p.net.n_edges) * p.ndof ** 2
        csr = (p.n_dof + 1) * 8 + nnz_k * 12
        e2e = {"value": len(ht) / (sum(ht) / 1e3), "unit": "solves/s",
               "h2d_bytes_per_step": int(h2d + csr), "d2h_bytes_per_step": int(csr + p.n_dof * 8)}
    return dict(times=times, last=last, prof=prof, launches=l1 - l0, clocks=clk, e2e=e2e,
                desc=desc, t_wall=t_wall, prof_steps=len(ptimes), prof_ms=sum(ptimes))


def cpu_oracle_sample(problem, iters_full, sample_iters=3):
    """Bounded CPU sample: the oracle's set-up plus a few PCG iterations.

    Returns (seconds for one full solve, extrapolated as set-up + iters_full x
    the measured time per iteration, description).
    """
    from oracle.solve import OracleSolver

    t0 = time.perf_counter()
    S = OracleSolver(problem)
    t1 = time.perf_counter()
    S.solve(rtol=1e-30, maxit=sample_iters)
    t2 = time.perf_counter()
    per_it = (t2 - t1) / sample_iters
    full = (t1 - t0) + iters_full * per_it
    desc = (f"oracle set-up ({t1 - t0:.1f} s) + {sample_iters} PCG iterations ({per_it:.2f} s each), "
            f"extrapolated to {iters_full} iterations")
    return full, desc


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "gb300":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    gen, desc = WORKLOADS[args.workload]
    if args.impl == "reference":
        if rank != 0:
            return
        prob = gen(0)
        iters = REF_ITERS.get(args.workload)
        times, desc_s = [], ""
        for k in range(args.warmup + args.steps):
            t, desc_s = cpu_oracle_sample(prob, iters)
            if k >= args.warmup:
                times.append(t)
        v = len(times) / sum(times)
        line = {
            "impl": "reference", "metric": "solves/s at rel-res 1e-8", "value": v, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "solve": "assembly+setup+pcg, rtol 1e-8", "impl": "cpu fp64 oracle"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"per step: {desc_s} ({desc}, numpy/scipy FP64)"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return
    r = run_gb300(args, rank, world, local)
    times = r["times"]
    tot = sum(times) / 1e3
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([tot], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    value = world * len(times) / tot
    oi, pi, st, kb = r["last"]
    prof = r["prof"]
    # dominant iteration kernel by device time inside the timed region
    cand = {k: v for k, v in prof.items() if k in kb and v[0] > 0}
    dom = max(cand, key=lambda k: cand[k][1]) if cand else None
    peak, src = peaks()
    roof = None
    if dom:
        n_l, ms = prof[dom]
        avg_s = ms / n_l / 1e3
        achieved = kb[dom] / avg_s / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "measured_in": "profiled pass of the same steps (CUDA events per launch)",
                "peak_source": src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None, "bytes_per_launch": int(kb[dom]), "avg_launch_us": round(avg_s * 1e6, 3)}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        t, desc_s = cpu_oracle_sample(WORKLOADS[args.workload][0](0), int(st.iterations))
        cpu = {"value": 1.0 / t, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{desc_s}; {desc}, numpy/scipy FP64"}
    if rank != 0:
        return
    share = {k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items() if v[0] > 0}
    share["profiled_pass"] = {"steps": r["prof_steps"], "ms": round(r["prof_ms"], 3),
                              "note": "eager launches, each timed with CUDA events"}
    line = {
        "metric": "solves/s at rel-res 1e-8", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": r["desc"], "precision": args.precision, "n_free": int(oi.n_free),
                   "nnz": int(oi.nnz_ff), "m0": int(pi.m0), "stars": int(pi.n_stars),
                   "sum_star": int(pi.sum_star), "factor_nnz": int(pi.factor_nnz),
                   "max_star": int(pi.max_star), "total_levels": int(pi.total_levels),
                   "max_levels": int(pi.max_levels), "setup_ms_last": round(pi.setup_ms, 3),
                   "iterations": int(st.iterations), "relres": st.relres,
                   "l2": "512 MiB buffer written between steps (outside the timed events)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"], "kernels": share,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
