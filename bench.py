"""Benchmark of the aTTN H_eff hot path on GB300.

Workload: 32x32 square-lattice TFIM (h = 3.04, open boundaries), binary TTN
with m = 128, disentanglers placed by the rule of Sec. 6.1 (256 requested),
H' = D^T H D split into rank-1 products. The timed unit is the local
eigensolve of the top [128,128,128] tensor: Lanczos (depth 20) whose H_eff
matvecs run in BF16 on the tensor cores (tcgen05, FP32 accumulation) with the
FP64 Krylov recurrence, reorthogonalisation and tridiagonal Ritz solve on the
GPU. The effective operators have the exact product structure of that node
(pair counts per link pair, three-link products, internal operators) taken
from the library's own term bookkeeping; their values are seeded synthetic
symmetric matrices (the cost does not depend on them).

metric: H_eff matvecs/s at m = 128 (whole job, all ranks); one step = one
Lanczos eigensolve (20 matvecs). N > 1 runs independent replicas (the path
is single-GPU; no collective on the data path).

--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded sample (a subset of the node's products), scaled to matvecs/s.
"""
import argparse
import hashlib
import json
import math
import re
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L, H_FIELD, M, N_DE, DEPTH = 32, 3.04, 128, 256, 20
WORKLOAD = "tfim32x32_m128_top_node_lanczos"


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, world, device):
    """The largest of every rank's value: a timed region ends when its slowest replica does."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units of all replicas per second over the (max-over-ranks) timed region."""
    return units_per_rank * world / (ms / 1000.0)


KERNEL_PROFILE = os.path.join(ROOT, "profiles", "sandwich_tc_kernel_tfim32x32_m128.md")


def kernel_source_sha():
    """SHA-256 of the sandwich kernel's source section: the code an ncu capture measured."""
    with open(os.path.join(ROOT, "paper_2507_21236_gb300", "csrc", "heff_tc.cu")) as f:
        src = f.read()
    a = src.index("// ------------------------------------------------------------------ kernel")
    b = src.index("// ------------------------------------------------------------ prep kernels")
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def profiled_traffic():
    """DRAM bytes (read + write) per launch from the committed ncu summary of the
    sandwich kernel, or None when the kernel's source has changed since the capture."""
    try:
        with open(KERNEL_PROFILE) as f:
            text = f.read()
    except OSError:
        return None
    sha = re.search(r"kernel source sha256: `?([0-9a-f]{64})", text)
    traffic = re.search(r"traffic per launch: `?([0-9]+)`? bytes", text)
    if not sha or not traffic or sha.group(1) != kernel_source_sha():
        return None
    return int(traffic.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def node_structure():
    """Product counts of the top node from the library (host bookkeeping)."""
    import torch
    from inputs import raw_tree_tensors
    from paper_2507_21236_gb300 import attn

    ctx = attn.attn_create(attn.attn_config_default(), torch.cuda.current_stream().cuda_stream)
    model = attn.attn_model_tfim(ctx, L, H_FIELD)
    # The placement rule gives the same disentanglers for every m in [16, 255]
    # on 32x32 (a pair is allowed when its lowest common tensor is at layer >= 4),
    # and the product bookkeeping does not depend on m: query it on an m = 16 tree.
    m_s = 16
    n = L * L
    nL = n.bit_length() - 2
    cap = lambda e: m_s if e >= 5 else min(2 ** (2 ** e), m_s)
    shapes = []
    for l in range(1, nL + 1):
        cd = 2 if l == 1 else cap(l - 1)
        pd = cap(l) if l < nL else cap(nL)
        shapes += [(cd, cd, pd)] * (n >> l)
    st = attn.attn_state_create(ctx, model, m_s, raw_tree_tensors(shapes, 0))
    n_de = attn.attn_de_place(st, N_DE)
    # optimised disentanglers are generic orthogonal matrices: use seeded ones so
    # that the mapped terms have the bond dimensions of a running aTTN (Sec. 4.3)
    from inputs import normal
    for k in range(n_de):
        q, r = np.linalg.qr(normal(11, 5000 + k, 16).reshape(4, 4))
        attn.attn_de_set(st, k, q * np.sign(np.diag(r)))
    attn.attn_map_hamiltonian(st)
    n_terms, n_prod = attn.attn_hamiltonian_info(st)
    nn, _, nl = attn.attn_state_info(st)
    top = nn - 2
    counts = attn.attn_heff_counts(st, top)
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(model)
    return ctx, {"n_de": n_de, "n_terms": n_terms, "n_products": n_prod, "node": top, "counts": counts}


def make_heff(attn, ctx, counts, seed=0):
    import torch
    from inputs import random_operators

    dev = lambda a: torch.as_tensor(a, device="cuda")
    h_int = [dev(random_operators(1, M, seed, 10 + s)[0]) for s in range(3)]
    pairs = {}
    for k in range(3):
        if counts[k]:
            pairs[k] = (dev(random_operators(counts[k], M, seed, 20 + 2 * k)),
                        dev(random_operators(counts[k], M, seed, 21 + 2 * k)))
    trip = None
    if counts[3]:
        trip = tuple(dev(random_operators(counts[3], M, seed, 40 + s)) for s in range(3))
    H = attn.attn_heff_create(ctx, (M, M, M), h_int, pairs, trip)
    return H, (h_int, pairs, trip)


def oracle_node_structure():
    """Product counts of the top node from the oracle's own placement, mapping and
    rank-1 split (no library code): pairs (0,1), (0,2), (1,2), triple, internal."""
    from inputs import normal
    from oracle.disentangle import map_terms, place_disentanglers, products_of
    from oracle.lattice import square_lattice, tfim_terms
    from oracle.tree import Tree

    terms = tfim_terms(square_lattice(L), H_FIELD)
    tree = Tree(L * L, 16)  # the placement rule gives the same pairs for every m in [16, 255]
    des = place_disentanglers(tree, terms, N_DE)
    us = []
    for k in range(len(des)):
        q, r = np.linalg.qr(normal(11, 5000 + k, 16).reshape(4, 4))
        us.append(q * np.sign(np.diag(r)))
    top = tree.top_nodes()[0]
    regions = [set(tree.region(top, s)) for s in range(3)]
    counts = [0] * 5
    slot_of_mask = {3: 0, 5: 1, 6: 2, 7: 3}
    for sites, _, _ in products_of(map_terms(terms, des, us)):
        mask = 0
        for x in sites:
            for k in range(3):
                if x in regions[k]:
                    mask |= 1 << k
        counts[slot_of_mask.get(mask, 4)] += 1
    return counts


def oracle_sample(budget_s, counts):
    """FP64 oracle H_eff on this process's host threads: the median time of single
    pair products of the [128]^3 top node (random operators; the cost does not depend
    on their values), scaled to the node's product list."""
    from inputs import random_operators, random_vector
    from oracle.ttn import heff_apply_ops

    x = random_vector((M, M, M), 1)
    total = counts[0] + counts[1] + counts[2]
    kinds = [(0, 1), (0, 2), (1, 2)]
    per_kind = {}
    t0 = time.perf_counter()
    done = 0
    while (time.perf_counter() - t0 < budget_s or done < 3) and done < total:
        k = done % 3
        a = random_operators(1, M, 7, 100 + done)
        b = random_operators(1, M, 7, 200 + done)
        t1 = time.perf_counter()
        heff_apply_ops(x, (None, None, None), {kinds[k]: (a, b)})
        per_kind.setdefault(k, []).append(time.perf_counter() - t1)
        done += 1
    med_all = statistics.median(sum(per_kind.values(), []))
    est = sum(counts[k] * statistics.median(per_kind.get(k, [med_all])) for k in range(3))
    est += counts[3] * 1.5 * med_all  # a three-link product: three mode products instead of two
    return {"value": 1.0 / est, "products_timed": done, "products_total": total}


def cpu_baseline(counts, budget_s=15.0):
    """The oracle timed on the host cores, single-threaded and with every core (the BLAS
    thread count is fixed in a child process before numpy loads)."""
    out = {}
    for threads in (1, os.cpu_count() or 1):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
                   MKL_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--mode", "oracle_sample",
                            "--sample-s", str(budget_s), "--counts", ",".join(map(str, counts))],
                           env=env, capture_output=True, text=True, check=True)
        out[threads] = json.loads(r.stdout.strip().splitlines()[-1])
    cores = max(out)
    return {"value": out[cores]["value"], "unit": "matvec/s", "cores": cores, "kind": "oracle",
            "single_thread_value": out[1]["value"],
            "sample": f"{out[cores]['products_timed']} of {out[cores]['products_total']} pair products of the "
                      f"[128]^3 top-node H_eff applied one by one by the FP64 oracle (numpy) in about "
                      f"{budget_s:.0f} s per thread count; the median time per product scaled to the node's "
                      f"full product list (counts from the oracle's own placement and mapping)"}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    counts = oracle_node_structure()
    budget = max(2.0, 20.0 / max(args.steps + args.warmup, 1))
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(oracle_sample(budget, counts)["value"])
    vals = vals[args.warmup:]
    v = statistics.median(vals)
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": "H_eff matvecs/s at m=128", "value": v, "unit": "matvec/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "model": "tfim", "L": L, "m": M,
                                            "node_counts_pairs01_02_12_triple_internal": counts},
            "cpu_baseline": {"value": v, "unit": "matvec/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step: about {budget:.1f} s of single pair products of the [128]^3 "
                                       f"top-node H_eff applied by the FP64 oracle (numpy, default BLAS threads), "
                                       f"median time per product scaled to the oracle's own product list"},
            "e2e": {"value": v, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mixed_solve_record(attn, ctx, H, x0, torch):
    """One accuracy-bearing mixed solve of the timed node against the FP64 solve."""
    stream = torch.cuda.current_stream()
    base = attn.attn_get_config(ctx)
    out = {}
    for name, upd in (("f64_split", {"matvec_dtype": attn.ATTN_F64, "f64_split": 1, "refine_steps": 0}),
                      ("mixed_split", {"matvec_dtype": attn.ATTN_BF16, "f64_split": 1, "refine_steps": 3,
                                       "refine_inner": 16, "refine_tol": 1e-10})):
        cfg = attn.attn_get_config(ctx)
        for k, v in upd.items():
            setattr(cfg, k, v)
        cfg.use_graphs = 0
        cfg.lanczos_tol = 1e-13
        attn.attn_set_config(ctx, cfg)
        T = x0.clone()
        attn.attn_eigsolve(H, T.data_ptr())  # warm-up (tensor-core tuning, split workspaces)
        T = x0.clone()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        theta, iters = attn.attn_eigsolve(H, T.data_ptr())
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms": a.elapsed_time(b), "theta": theta, "matvecs": iters}
    # converged FP64 reference: split-FP64 Lanczos of depth 60, restarted from its own result
    cfg = attn.attn_get_config(ctx)
    cfg.matvec_dtype, cfg.f64_split, cfg.refine_steps, cfg.use_graphs = attn.ATTN_F64, 1, 0, 0
    cfg.lanczos_depth, cfg.lanczos_tol = 60, 1e-14
    attn.attn_set_config(ctx, cfg)
    T = x0.clone()
    for _ in range(4):
        th_ref, _ = attn.attn_eigsolve(H, T.data_ptr())
    attn.attn_set_config(ctx, base)
    out["converged_f64_theta"] = th_ref
    for name in ("f64_split", "mixed_split"):
        out[name]["rel_diff_vs_converged"] = (out[name]["theta"] - th_ref) / abs(th_ref)
    out["note"] = ("one local solve from the same start: depth-20 Lanczos with FP64 (split) matvecs, and BF16 "
                   "matvecs + 3 FP64 Rayleigh-Ritz refinements with BF16 Jacobi-Davidson inner solves; "
                   "reference: 4 restarts of a depth-60 split-FP64 Lanczos")
    return out


SWEEP_L, SWEEP_M, SWEEP_N = 16, 128, 2


def sweep_record(attn, torch):
    """16x16 TFIM (h = 3.04), m = 128: the first two aTTN sweeps (S_TTN = 1, then
    disentangler updates) of the FP64 path (contractions as split BF16 products) and
    of the mixed paths (BF16 or TF32 Lanczos + FP64 refinement), from the same tensors."""
    from inputs import raw_tree_tensors

    n = SWEEP_L * SWEEP_L
    raw = raw_tree_tensors(tree_shapes(n, SWEEP_M), 0)
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    for name in ("f64_split", "mixed_split", "mixed_tf32_split"):
        cfg = arm_config(attn, name)
        ctx = attn.attn_create(cfg, stream)
        model = attn.attn_model_tfim(ctx, SWEEP_L, H_FIELD)
        st = attn.attn_state_create(ctx, model, SWEEP_M, raw)
        n_de = attn.attn_de_place(st, n // 4)
        es, ts = [], []
        for _ in range(SWEEP_N):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            es.append(attn.attn_sweep(st) / n)
            ts.append(time.perf_counter() - t0)
        out[name] = {"s_per_sweep": ts, "energy_per_site": es, "n_de": n_de}
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(model)
        attn.attn_destroy(ctx)
    for name in ("mixed_split", "mixed_tf32_split"):
        out[name]["minus_f64_per_site"] = [a - b for a, b in zip(out[name]["energy_per_site"],
                                                                  out["f64_split"]["energy_per_site"])]
    out["config"] = {"workload": f"tfim{SWEEP_L}x{SWEEP_L}_m{SWEEP_M}_first_{SWEEP_N}_sweeps", "s_ttn": 1,
                     "mixed_split": "bf16 Lanczos + <= 8 FP64 Rayleigh-Ritz corrections from 16-step bf16 CG "
                                    "Jacobi-Davidson solves until theta moves by < 1e-10 |theta|",
                     "mixed_tf32_split": "the same with TF32 matvecs",
                     "contractions": "FP64 contractions as split bf16 products (f64_split) in every arm"}
    return out


def precision_arms(attn):
    """Configuration overrides of each precision policy the sweep benchmarks compare."""
    # BF16 Lanczos, then FP64 Rayleigh-Ritz with BF16 Jacobi-Davidson corrections:
    # three of them (the library default), or until theta moves by < 1e-10 |theta|
    k3 = {"matvec_dtype": attn.ATTN_BF16, "refine_steps": 3, "refine_inner": 16}
    jd = {"matvec_dtype": attn.ATTN_BF16, "refine_steps": 8, "refine_inner": 16, "refine_tol": 1e-10}
    # *_split: FP64 contractions as exact BF16 slice products on the tensor cores
    tf = dict(jd, matvec_dtype=attn.ATTN_TF32)
    return {"f64": {}, "mixed_k3": k3, "mixed": jd, "f64_split": {"f64_split": 1},
            "mixed_tf32_split": dict(tf, f64_split=1),
            "mixed_k3_split": dict(k3, f64_split=1), "mixed_split": dict(jd, f64_split=1),
            "mixed_split_t12": dict(jd, f64_split=1, refine_tol=1e-12)}


PROFILE_IDS = {0: "tc_heff_kernel", 1: "fp64_gemm", 2: "tc_gemm", 3: "split_fp64_gemm", 4: "centre_moves",
               5: "heff_builds", 6: "lanczos", 7: "fp64_energy_refinement", 8: "de_updates"}


def profile_report(attn, ctx, nsweeps):
    """Stream time per sweep of the library's kernels and local-step phases (attn_profile_read)."""
    out = {}
    for kid, name in PROFILE_IDS.items():
        ms, n, _ = attn.attn_profile_read(ctx, kid)
        if n:
            out[name] = {"ms_per_sweep": ms / max(nsweeps, 1), "count_per_sweep": n / max(nsweeps, 1)}
    return out


def arm_config(attn, name):
    cfg = attn.attn_config_default()
    for k, v in precision_arms(attn)[name].items():
        setattr(cfg, k, v)
    return cfg


def run_sweeps(args):
    """Sweep time to dE/site <= 1e-8: FP64 matvecs vs BF16 matvecs + FP64 refinement,
    same aTTN schedule (S_TTN = 1) from identical inputs, on one GPU."""
    import torch
    from __graft_entry__ import build
    from inputs import raw_tree_tensors
    from paper_2507_21236_gb300 import attn

    build()
    Ls, ms, h = args.sweep_L, args.sweep_m, H_FIELD
    n = Ls * Ls
    nL = n.bit_length() - 2
    cap = lambda e: ms if e >= 5 else min(2 ** (2 ** e), ms)
    shapes = []
    for l in range(1, nL + 1):
        cd = 2 if l == 1 else cap(l - 1)
        pd = cap(l) if l < nL else cap(nL)
        shapes += [(cd, cd, pd)] * (n >> l)
    raw = raw_tree_tensors(shapes, 0)
    out = {}
    modes = args.sweep_arms.split(",")
    ref = modes[0]  # the FP64 arm the others are compared with
    assert ref in ("f64", "f64_split"), "the first arm is the FP64 reference"
    for mode in modes:
        cfg = arm_config(attn, mode)
        cfg.compress_terms = 1 if args.compress else 0
        ctx = attn.attn_create(cfg, torch.cuda.current_stream().cuda_stream)
        if args.model == "tri_heisenberg":
            model = attn.attn_model_tri_heisenberg(ctx, Ls, 1.0)
        else:
            model = attn.attn_model_tfim(ctx, Ls, h)
        st = attn.attn_state_create(ctx, model, ms, raw)
        n_de = attn.attn_de_place(st, n // 4)
        if args.phases:
            attn.attn_profile_enable(ctx, True)
        es, ts = [], []
        t_conv = None
        for s in range(args.max_sweeps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            es.append(attn.attn_sweep(st))
            ts.append(time.perf_counter() - t0)
            if s >= 2 and abs(es[-1] - es[-2]) / n <= 1e-8 and t_conv is None:
                t_conv = (s + 1, sum(ts))
                break
        out[mode] = {"energies_per_site": [e / n for e in es], "sweep_s": ts,
                     "sweeps_to_1e-8": t_conv[0] if t_conv else None,
                     "time_to_1e-8_s": t_conv[1] if t_conv else None, "n_de": n_de}
        if args.phases:
            out[mode]["profile"] = profile_report(attn, ctx, len(es))
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(model)
        attn.attn_destroy(ctx)
    d = {k: abs(out[k]["energies_per_site"][-1] - out[ref]["energies_per_site"][-1]) for k in out if k != ref}
    head = next((k for k in ("mixed_split_t12", "mixed_split", "mixed", "mixed_k3") if k in out), ref)
    line = {"metric": "sweep time to dE/site<=1e-8, mixed vs FP64", "unit": "s",
            "value": out[head]["time_to_1e-8_s"], "value_arm": head, "higher_is_better": False,
            "f64_value": out[ref]["time_to_1e-8_s"], "final_energy_per_site_diff": d,
            "config": {"workload": f"{args.model}{Ls}x{Ls}_m{ms}_sweeps", "L": Ls, "m": ms,
                       "coupling": 1.0 if args.model == "tri_heisenberg" else h, "compress_terms": bool(args.compress),
                       "s_ttn": 1, "lanczos_depth": 20,
                       "mixed": "bf16 Lanczos + <= 8 FP64 Rayleigh-Ritz corrections from 16-step bf16 CG "
                                "Jacobi-Davidson solves, until theta moves by < 1e-10 |theta|",
                       "mixed_k3": "bf16 Lanczos + 3 such corrections (library default)",
                       "_split": "FP64 contractions as exact bf16 slice products on the tensor cores (f64_split)"},
            "runs": out}
    print(json.dumps(line), flush=True)


def run_converge(args):
    """Converged energies under a frozen disentangler layer: one FP64 prefix of aTTN
    sweeps (S_TTN = 1, then disentangler updates), after which every precision arm
    starts from that identical state and H' and sweeps the TTN until the energy
    changes by <= 1e-8 per site; final energies are compared with the FP64 arm's."""
    import torch
    from __graft_entry__ import build
    from inputs import raw_tree_tensors
    from paper_2507_21236_gb300 import attn

    build()
    Ls, ms, h = args.sweep_L, args.sweep_m, H_FIELD
    n = Ls * Ls
    raw = raw_tree_tensors(tree_shapes(n, ms), 0)
    stream = torch.cuda.current_stream().cuda_stream

    arms = args.arms.split(",")
    ref = arms[0]  # the FP64 arm the others are compared with; it also runs the prefix
    assert ref in ("f64", "f64_split"), "the first arm is the FP64 reference"
    # FP64 prefix: sweep 1 without disentanglers, then args.prefix - 1 sweeps with updates
    ctx = attn.attn_create(arm_config(attn, ref), stream)
    model = attn.attn_model_tfim(ctx, Ls, h)
    st = attn.attn_state_create(ctx, model, ms, raw)
    n_de = attn.attn_de_place(st, n // 4)
    t0 = time.perf_counter()
    prefix_e = [attn.attn_sweep(st) / n for _ in range(args.prefix)]
    prefix_s = time.perf_counter() - t0
    nn, centre, _ = attn.attn_state_info(st)
    tensors = [attn.attn_node_get(st, i) for i in range(nn)]
    us = [attn.attn_de_get(st, k) for k in range(n_de)]
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(model)
    attn.attn_destroy(ctx)

    out = {}
    for name in arms:
        cfg = arm_config(attn, name)
        ctx = attn.attn_create(cfg, stream)
        model = attn.attn_model_tfim(ctx, Ls, h)
        st = attn.attn_state_create(ctx, model, ms, raw)
        assert attn.attn_de_place(st, n // 4) == n_de
        for k, u in enumerate(us):
            attn.attn_de_set(st, k, u)
        attn.attn_map_hamiltonian(st)
        attn.attn_move_centre(st, centre)
        for i, t in enumerate(tensors):
            attn.attn_node_set(st, i, t)
        es = [attn.attn_energy(st) / n]
        if args.phases:
            attn.attn_profile_enable(ctx, True)
        ts = []
        conv = None
        for s in range(args.max_sweeps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            es.append(attn.attn_ttn_sweep(st) / n)
            ts.append(time.perf_counter() - t0)
            if abs(es[-1] - es[-2]) <= 1e-8:
                conv = s + 1
                break
        out[name] = {"start_energy_per_site": es[0], "energies_per_site": es[1:], "sweep_s": ts,
                     "sweeps_to_1e-8": conv, "time_to_1e-8_s": sum(ts) if conv else None}
        if args.phases:
            out[name]["profile"] = profile_report(attn, ctx, len(ts))
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(model)
        attn.attn_destroy(ctx)
    e_ref = out[ref]["energies_per_site"][-1]
    head = next((k for k in ("mixed_tf32_split", "mixed_split_t12", "mixed_split", "mixed", "mixed_k3") if k in out),
                ref)
    line = {"metric": "time to dE/site<=1e-8 under a frozen disentangler layer, mixed vs FP64", "unit": "s",
            "value": out[head]["time_to_1e-8_s"], "value_arm": head, "higher_is_better": False,
            "f64_value": out[ref]["time_to_1e-8_s"], "f64_arm": ref,
            "final_energy_per_site_minus_f64": {k: out[k]["energies_per_site"][-1] - e_ref for k in out if k != ref},
            "config": {"workload": f"tfim{Ls}x{Ls}_m{ms}_converge", "L": Ls, "m": ms, "h": h, "n_de": n_de,
                       "prefix": f"{args.prefix} FP64 aTTN sweeps (S_TTN = 1, then disentangler updates), "
                                 f"{prefix_s:.1f} s, E/site {prefix_e}",
                       "lanczos_depth": 20,
                       "mixed_k3": "bf16 Lanczos + 3 FP64 Rayleigh-Ritz corrections from 16-step bf16 CG "
                                   "Jacobi-Davidson solves (library default)",
                       "mixed": "bf16 Lanczos + <= 8 such corrections, until theta moves by < 1e-10 |theta|",
                       "_t12": "refinement until theta moves by < 1e-12 |theta|",
                       "_split": "FP64 contractions (renormalisation, FP64 matvecs, environments) as exact bf16 "
                                 "slice products on the tensor cores (f64_split)"},
            "runs": out}
    print(json.dumps(line), flush=True)


def run_split(args):
    """FP64 H_eff applications of the 32x32 top node (m = 128, its real product
    counts, synthetic operators) with the FP64 contractions as exact BF16 slice
    products on the tensor cores, beside the same applications on FP64 FMAs."""
    import torch
    from __graft_entry__ import build
    from paper_2507_21236_gb300 import attn

    build()
    torch.cuda.set_device(0)
    ctx, info = node_structure()
    counts = info["counts"]
    H, _ = make_heff(attn, ctx, counts)
    stream = torch.cuda.current_stream()
    x = torch.randn((M, M, M), device="cuda", dtype=torch.float64, generator=torch.Generator(device="cuda").manual_seed(1))
    y = torch.empty_like(x)
    y64 = torch.empty_like(x)
    fl = attn.attn_heff_info(H)[2]
    out = {}
    for split in (1, 0):
        cfg = attn.attn_get_config(ctx)
        cfg.f64_split = split
        attn.attn_set_config(ctx, cfg)
        dst = y if split else y64
        attn.attn_heff_apply(H, x.data_ptr(), dst.data_ptr(), attn.ATTN_F64)  # warm-up
        attn.attn_profile_enable(ctx, True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = args.steps if split else 1
        a.record(stream)
        for _ in range(reps):
            attn.attn_heff_apply(H, x.data_ptr(), dst.data_ptr(), attn.ATTN_F64)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        prof = {name: attn.attn_profile_read(ctx, kid) for kid, name in ((1, "fp64_fma_gemm"), (3, "split_gemm"))}
        attn.attn_profile_enable(ctx, False)
        out["split" if split else "fma"] = {
            "ms_per_apply": ms, "tflops": fl / ms / 1e9,
            "kernels": {k: {"ms": v[0] / reps, "launches": v[1] / reps, "tflops": v[2] / max(v[0], 1e-9) / 1e9}
                        for k, v in prof.items() if v[1]}}
    err = float((y - y64).abs().max() / y64.abs().max())
    print(json.dumps({"metric": "FP64 H_eff apply, 32x32 top node, m=128", "unit": "ms",
                      "gflop_per_apply": fl / 1e9, "node_counts_pairs01_02_12_triple": list(counts[:4]),
                      "max_rel_diff_split_vs_fma": err, "runs": out}), flush=True)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)


def run_sttn(args):
    """The S_TTN study of Sec. 6.3 (Fig. benchmark-4deopt) at a size one GPU call affords:
    the same total number of sweeps, of which the first S_TTN run without disentangler
    optimisation and the rest update the disentangler layer every sweep; final energy
    per site and run time for each S_TTN."""
    import torch
    from __graft_entry__ import build
    from inputs import raw_tree_tensors
    from paper_2507_21236_gb300 import attn

    build()
    Ls, ms = args.sweep_L, args.sweep_m
    n = Ls * Ls
    raw = raw_tree_tensors(tree_shapes(n, ms), 0)
    stream = torch.cuda.current_stream().cuda_stream
    rows = []
    for s_ttn in [int(v) for v in args.sttn_values.split(",")]:
        # s_ttn = -1: the plain TTN at the same bond dimension (no disentanglers)
        cfg = arm_config(attn, args.sttn_arm)
        cfg.s_ttn = max(s_ttn, 0)
        ctx = attn.attn_create(cfg, stream)
        model = attn.attn_model_tfim(ctx, Ls, H_FIELD)
        st = attn.attn_state_create(ctx, model, ms, raw)
        n_de = attn.attn_de_place(st, n // 4 if s_ttn >= 0 else 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        es = [attn.attn_sweep(st) / n for _ in range(args.max_sweeps)]
        rows.append({"s_ttn": s_ttn, "energy_per_site": es, "final": es[-1], "s": time.perf_counter() - t0,
                     "n_de": n_de})
        print(json.dumps(rows[-1]), flush=True)
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(model)
        attn.attn_destroy(ctx)
    best = min(rows, key=lambda r: r["final"])
    print(json.dumps({"metric": "final energy per site vs S_TTN (fixed total sweeps)", "unit": "E/site",
                      "best_s_ttn": best["s_ttn"], "config": {"workload": f"tfim{Ls}x{Ls}_m{ms}_sttn", "L": Ls,
                      "m": ms, "h": H_FIELD, "sweeps": args.max_sweeps, "arm": args.sttn_arm}, "runs": rows}),
          flush=True)


def train_learned_start(attn, ctx, torch):
    """MLP of the learned disentangler start, trained on the (two-site density matrix at
    the first update, final disentangler) pairs of plain 8x8 (seeds 0-3) and 16x16
    (seeds 0-1) TFIM runs at m = 16 (three aTTN sweeps each)."""
    from inputs import raw_tree_tensors
    from oracle.mlp import init_params

    rhos, targets = [], []
    for Ls, seeds in ((8, range(4)), (16, range(2))):
        for seed in seeds:
            model = attn.attn_model_tfim(ctx, Ls, H_FIELD)
            st = attn.attn_state_create(ctx, model, 16, raw_tree_tensors(tree_shapes(Ls * Ls, 16), seed))
            n = attn.attn_de_place(st, Ls * Ls // 4)
            for _ in range(3):
                attn.attn_sweep(st)
            r, u = attn.attn_de_training_pairs(st, n)
            rhos.append(r)
            targets.append(u)
            attn.attn_state_destroy(st)
            attn.attn_model_destroy(model)
    p = init_params(0)
    flat = np.concatenate([p[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)
    mlp = attn.attn_mlp_create(ctx, flat)
    rho, ut = np.concatenate(rhos), np.concatenate(targets)
    l0, _ = attn.attn_mlp_loss_grad(mlp, rho, ut)
    l1 = attn.attn_mlp_train(mlp, rho, ut, 600, 2e-3)
    return mlp, {"samples": int(rho.shape[0]), "loss_before": l0, "loss_after": l1}


def run_target(args):
    """The 32x32 TFIM aTTN at m = 128 (h = 3.04, 184 placed disentanglers), from one set
    of raw tensors: the FP64 path (contractions as split BF16 products), the mixed path
    (BF16 Lanczos + FP64 refinement, split contractions), and the mixed path with the
    learned disentangler start. Per sweep: wall time, energy per site, its change, and
    the mixed arms' difference to FP64."""
    import torch
    from __graft_entry__ import build
    from inputs import raw_tree_tensors
    from paper_2507_21236_gb300 import attn

    build()
    Ls, ms = args.sweep_L, args.sweep_m
    n = Ls * Ls
    raw = raw_tree_tensors(tree_shapes(n, ms), 0)
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    arms = args.arms.split(",")
    for name in arms:
        learned = name.endswith("+learned")
        cfg = arm_config(attn, name.replace("+learned", ""))
        ctx = attn.attn_create(cfg, stream)
        mlp = None
        if learned:
            mlp, out["learned_training"] = train_learned_start(attn, ctx, torch)
        model = attn.attn_model_tfim(ctx, Ls, H_FIELD)
        st = attn.attn_state_create(ctx, model, ms, raw)
        n_de = attn.attn_de_place(st, n // 4)
        if mlp is not None:
            attn.attn_set_learned_init(st, mlp)
        es, ts, ek = [], [], []
        for s in range(args.max_sweeps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            es.append(attn.attn_sweep(st) / n)
            ts.append(time.perf_counter() - t0)
            if n_de and s >= 1:  # this sweep's disentangler update: sum_k E_k of its start and its result
                e = attn.attn_de_energies(st, n_de)
                ek.append([float(e[:, 0].sum()), float(e[:, 1].sum())])
            print(json.dumps({"arm": name, "sweep": s + 1, "s": ts[-1], "energy_per_site": es[-1],
                              "sum_Ek_update": ek[-1] if ek and s >= 1 else None}), flush=True)
        rec = {"s_per_sweep": ts, "energy_per_site": es, "delta_per_site": [b - a for a, b in zip(es[:-1], es[1:])],
               "n_de": n_de, "sum_Ek_per_update_start_result": ek}
        if mlp is not None:
            rec["learned_used_fallback"] = list(attn.attn_learned_init_report(st))
            attn.attn_mlp_destroy(mlp)
        out[name] = rec
        attn.attn_state_destroy(st)
        attn.attn_model_destroy(model)
        attn.attn_destroy(ctx)
    ref = out.get(arms[0])
    for name in arms[1:]:
        out[name]["minus_" + arms[0] + "_per_site"] = [a - b for a, b in zip(out[name]["energy_per_site"],
                                                                              ref["energy_per_site"])]
    print(json.dumps({"metric": "aTTN sweeps, 32x32 TFIM m=128: time per sweep and energy per site by arm",
                      "config": {"workload": f"tfim{Ls}x{Ls}_m{ms}_target", "L": Ls, "m": ms, "h": H_FIELD,
                                 "s_ttn": 1, "arms": arms}, "runs": out}), flush=True)


# (name, model, L, m, coupling): the matvec benchmark shapes of every configuration
NODE_CONFIGS = [("C2", "tfim", 8, 32, 3.04), ("C3", "tfim", 16, 64, 3.04), ("C3", "tfim", 16, 128, 3.04),
                ("C4", "heis", 16, 64, 1.0), ("C4", "heis", 16, 128, 1.0), ("C5", "tfim", 32, 128, 3.04)]


def tree_shapes(n, m):
    """[child, child, parent] shapes of the binary tree over n sites, layer by layer."""
    nL = n.bit_length() - 2
    cap = lambda e: m if e >= 5 else min(2 ** (2 ** e), m)
    shapes = []
    for l in range(1, nL + 1):
        cd = 2 if l == 1 else cap(l - 1)
        pd = cap(l) if l < nL else cap(nL)
        shapes += [(cd, cd, pd)] * (n >> l)
    return shapes


def config_counts(attn, ctx, model_kind, Ls, coupling):
    """Per-node product counts of a configuration after mapping through seeded
    random orthogonal disentanglers (the bookkeeping is the same for every m in
    [16, 255], so it is queried on an m = 16 tree)."""
    from inputs import normal, raw_tree_tensors

    n = Ls * Ls
    model = (attn.attn_model_tfim(ctx, Ls, coupling) if model_kind == "tfim"
             else attn.attn_model_tri_heisenberg(ctx, Ls, coupling))
    st = attn.attn_state_create(ctx, model, 16, raw_tree_tensors(tree_shapes(n, 16), 0))
    n_de = attn.attn_de_place(st, n // 4)
    for k in range(n_de):
        q, r = np.linalg.qr(normal(11, 5000 + k, 16).reshape(4, 4))
        attn.attn_de_set(st, k, q * np.sign(np.diag(r)))
    attn.attn_map_hamiltonian(st)
    nn = attn.attn_state_info(st)[0]
    counts = [attn.attn_heff_counts(st, i) for i in range(nn)]
    attn.attn_state_destroy(st)
    attn.attn_model_destroy(model)
    return n_de, counts


def run_nodes(args):
    """H_eff apply time of every [m,m,m] node of each configuration, BF16 tensor-core
    path (all nodes) and FP64 path (a sample), with the nodes' real product counts."""
    import torch
    from __graft_entry__ import build
    from paper_2507_21236_gb300 import attn

    build()
    torch.cuda.set_device(0)
    ctx = attn.attn_create(attn.attn_config_default(), torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(0)
    stream = torch.cuda.current_stream()
    out = []

    def timed_apply(H, x, y, dt, reps):
        attn.attn_heff_apply(H, x.data_ptr(), y.data_ptr(), dt)  # warm-up (first BF16 call builds and tunes)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            attn.attn_heff_apply(H, x.data_ptr(), y.data_ptr(), dt)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    for name, kind, Ls, m, coupling in NODE_CONFIGS:
        n_de, counts = config_counts(attn, ctx, kind, Ls, coupling)
        shapes = tree_shapes(Ls * Ls, m)
        big = [i for i, sh in enumerate(shapes) if sh == (m, m, m)]
        rmax = max(max(counts[i][:4]) for i in big)
        pool = torch.randn((2, rmax, m, m), device="cuda", dtype=torch.float64, generator=gen) / math.sqrt(m)
        hint = [torch.randn((m, m), device="cuda", dtype=torch.float64, generator=gen) / math.sqrt(m) for _ in range(3)]
        x = torch.randn((m, m, m), device="cuda", dtype=torch.float64, generator=gen)
        y = torch.empty_like(x)
        rows, by_counts = [], {}
        for i in big:
            c = counts[i]
            key = tuple(c[:4])
            if key not in by_counts:
                pairs = {k: (pool[0, :c[k]], pool[1, :c[k]]) for k in range(3) if c[k]}
                trip = tuple(pool[s % 2, :c[3]] for s in range(3)) if c[3] else None
                H = attn.attn_heff_create(ctx, (m, m, m), hint, pairs, trip)
                fl = attn.attn_heff_info(H)[2]
                ms = timed_apply(H, x, y, attn.ATTN_BF16, 5)
                ms_tf = timed_apply(H, x, y, attn.ATTN_TF32, 5)
                by_counts[key] = (fl, ms, H, ms_tf)
            fl, ms, _, ms_tf = by_counts[key]
            rows.append({"node": i, "counts": list(c[:4]), "gflop": fl / 1e9, "bf16_ms": ms, "tf32_ms": ms_tf})
        # FP64 on a sample: the lightest, the median and the heaviest node
        srt = sorted(rows, key=lambda r: r["gflop"])
        sample = [srt[0], srt[len(srt) // 2], srt[-1]]
        for r in sample:
            H = by_counts[tuple(r["counts"])][2]
            r["f64_ms"] = timed_apply(H, x, y, attn.ATTN_F64, 1)
        # error of each low precision against FP64 on the heaviest node (normwise, max-abs)
        H = by_counts[tuple(srt[-1]["counts"])][2]
        y64 = torch.empty_like(x)
        attn.attn_heff_apply(H, x.data_ptr(), y64.data_ptr(), attn.ATTN_F64)
        errs = {}
        for dname, dt in (("bf16", attn.ATTN_BF16), ("tf32", attn.ATTN_TF32)):
            attn.attn_heff_apply(H, x.data_ptr(), y.data_ptr(), dt)
            torch.cuda.synchronize()
            errs[dname] = float((y - y64).abs().max() / y64.abs().max())
        # the same FP64 applications with the contractions as exact BF16 slice products
        cfg = attn.attn_get_config(ctx)
        cfg.f64_split = 1
        attn.attn_set_config(ctx, cfg)
        for r in sample:
            H = by_counts[tuple(r["counts"])][2]
            r["f64_split_ms"] = timed_apply(H, x, y, attn.ATTN_F64, 3)
        cfg.f64_split = 0
        attn.attn_set_config(ctx, cfg)
        for _, _, H, _ in by_counts.values():
            attn.attn_heff_destroy(H)
        del pool
        tot_fl = sum(r["gflop"] for r in rows)
        tot_bf = sum(r["bf16_ms"] for r in rows)
        f64_fl = sum(r["gflop"] for r in sample)
        f64_ms = sum(r["f64_ms"] for r in sample)
        out.append({"config": name, "model": kind, "L": Ls, "m": m, "n_de_placed": n_de, "nodes": len(rows),
                    "products_per_node": [min(sum(r["counts"]) for r in rows), max(sum(r["counts"]) for r in rows)],
                    "gflop_per_matvec": [round(srt[0]["gflop"], 2), round(srt[-1]["gflop"], 2)],
                    "bf16": {"ms_all_nodes": round(tot_bf, 3), "tflops_flop_weighted": tot_fl / tot_bf,
                             "tflops_top": rows[-1]["gflop"] / rows[-1]["bf16_ms"],
                             "max_rel_err_vs_f64_heaviest": errs["bf16"]},
                    "tf32": {"ms_all_nodes": round(sum(r["tf32_ms"] for r in rows), 3),
                             "tflops_flop_weighted": tot_fl / sum(r["tf32_ms"] for r in rows),
                             "tflops_top": rows[-1]["gflop"] / rows[-1]["tf32_ms"],
                             "max_rel_err_vs_f64_heaviest": errs["tf32"]},
                    "f64_sample": {"nodes": [r["node"] for r in sample],
                                   "ms": [round(r["f64_ms"], 3) for r in sample],
                                   "tflops_flop_weighted": f64_fl / f64_ms,
                                   "split_ms": [round(r["f64_split_ms"], 3) for r in sample],
                                   "split_tflops_flop_weighted": f64_fl / sum(r["f64_split_ms"] for r in sample)},
                    "bf16_speedup_on_sample": f64_ms / sum(r["bf16_ms"] for r in sample)})
        print(json.dumps(out[-1]), flush=True)
    print(json.dumps({"metric": "H_eff apply per [m,m,m] node, BF16 and TF32 tensor cores vs FP64",
                      "unit": "TFLOP/s", "configs": out}), flush=True)
    attn.attn_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="matvec",
                    choices=["matvec", "sweep", "nodes", "converge", "split", "sttn", "target", "oracle_sample"])
    ap.add_argument("--sweep-L", type=int, default=16)
    ap.add_argument("--sweep-m", type=int, default=32)
    ap.add_argument("--model", default="tfim", choices=["tfim", "tri_heisenberg"],
                    help="sweep mode: square-lattice TFIM (h = 3.04) or triangular-lattice Heisenberg (J = 1)")
    ap.add_argument("--compress", action="store_true", help="sweep mode: compress mapped terms on the same sites")
    ap.add_argument("--max-sweeps", type=int, default=30)
    ap.add_argument("--prefix", type=int, default=3, help="FP64 aTTN sweeps before the frozen-layer runs")
    ap.add_argument("--arms", default="f64,mixed_k3,mixed,mixed_split",
                    help="converge mode: comma-separated precision arms (f64 first)")
    ap.add_argument("--sweep-arms", default="f64,mixed,mixed_k3",
                    help="sweep mode: comma-separated precision arms (f64 first)")
    ap.add_argument("--sttn-values", default="-1,0,1,2,3,5",
                    help="sttn mode: S_TTN values to compare (-1: plain TTN, no disentanglers)")
    ap.add_argument("--sttn-arm", default="mixed_split", help="sttn mode: precision arm of every run")
    ap.add_argument("--phases", action="store_true",
                    help="sweep/converge modes: report stream time per kernel class and local-step phase "
                         "(event pairs around every launch: adds host overhead, keep off for timings)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="attn")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="matvec mode: skip the 16x16 m=128 sweep record")
    ap.add_argument("--no-solve", action="store_true",
                    help="matvec mode: skip the mixed-precision local-solve record (profiling runs)")
    ap.add_argument("--sample-s", type=float, default=15.0, help=argparse.SUPPRESS)
    ap.add_argument("--counts", default="", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.mode == "oracle_sample":
        print(json.dumps(oracle_sample(args.sample_s, [int(c) for c in args.counts.split(",")])), flush=True)
        return
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "sweep":
        return run_sweeps(args)
    if args.mode == "nodes":
        return run_nodes(args)
    if args.mode == "converge":
        return run_converge(args)
    if args.mode == "split":
        return run_split(args)
    if args.mode == "sttn":
        return run_sttn(args)
    if args.mode == "target":
        return run_target(args)
    args.warmup = max(args.warmup, 3)

    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from __graft_entry__ import build
    from paper_2507_21236_gb300 import attn

    build()
    ctx, info = node_structure()
    counts = info["counts"]
    cfg = attn.attn_config_default()
    cfg.lanczos_depth = DEPTH
    cfg.lanczos_tol = 0.0  # fixed depth: every step runs the full 20 matvecs
    cfg.matvec_dtype = attn.ATTN_BF16
    cfg.refine_steps = 0
    cfg.use_graphs = 1  # each eigensolve replays one captured CUDA graph
    attn.attn_set_config(ctx, cfg)
    H, keep = make_heff(attn, ctx, counts)
    npair, ntrip, flops_mv = attn.attn_heff_info(H)
    from inputs import random_vector
    x0 = torch.as_tensor(random_vector((M, M, M), 3), device="cuda")
    T = torch.empty_like(x0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        T.copy_(x0)
        theta, iters = attn.attn_eigsolve(H, T.data_ptr())
        return iters

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    evs = []
    l0 = attn.attn_kernel_launches(ctx)
    attn.attn_profile_enable(ctx, True)
    iters_total = 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()  # the timed region is what an external profiler captures
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            iters_total += step()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    launches = attn.attn_kernel_launches(ctx) - l0
    k_ms, k_n, k_fl = attn.attn_profile_read(ctx, 0)
    attn.attn_profile_enable(ctx, False)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world, "cuda")
    value = whole_job_rate(iters_total, world, ms)

    # end to end through the C ABI on host buffers: every step one attn_eigsolve_host
    # call copies the start tensor in, solves and copies the Ritz vector back
    host_T = torch.empty(x0.shape, dtype=torch.float64).pin_memory()
    host_np = host_T.numpy()
    x0_host = x0.cpu().numpy()
    torch.cuda.synchronize()
    e_iters = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host_np[...] = x0_host
        theta, it = attn.attn_eigsolve_host(H, host_np)
        e_iters += it
    e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0, world, "cuda")
    e2e = {"value": whole_job_rate(e_iters, world, e_ms), "unit": "matvec/s",
           "h2d_bytes_per_step": int(x0.numel() * 8), "d2h_bytes_per_step": int(x0.numel() * 8 + 8),
           "call": "attn_eigsolve_host (pinned host tensor in and out, host wall clock)"}

    # the accuracy-bearing form of the same solve: BF16 Lanczos then FP64 Rayleigh-Ritz
    # refinement (3 Jacobi-Davidson corrections, FP64 contractions as split BF16 products)
    # the same timed loop with the optional FP32 Krylov basis (lanczos_basis = 1): the
    # reorthogonalisation in FP32 instead of FP64 (not the default precision policy)
    cfg_b = attn.attn_get_config(ctx)
    cfg_b.lanczos_basis = 1
    attn.attn_set_config(ctx, cfg_b)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs_b, it_b = [], 0
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        it_b += step()
        b.record(stream)
        evs_b.append((a, b))
    torch.cuda.synchronize()
    ms_b = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs_b), world, "cuda")
    cfg_b.lanczos_basis = 0
    attn.attn_set_config(ctx, cfg_b)
    f32_basis = {"value": whole_job_rate(it_b, world, ms_b), "unit": "matvec/s", "ms_per_step": ms_b / args.steps,
                 "config": "lanczos_basis = 1: Krylov basis and CGS2 reorthogonalisation in FP32 (recurrence "
                           "scalars, matvec vectors and Ritz vector FP64); an option, not the default policy"}

    solve = None if args.no_solve else mixed_solve_record(attn, ctx, H, x0, torch)

    peaks, src = measured_peaks()
    achieved = (k_fl / k_n) / ((k_ms / k_n) / 1000.0) / 1e12 if k_n else None
    peak = peaks["bf16_tflops"]
    traffic = profiled_traffic()
    roof = {"bound": "tensor", "kernel": "sandwich_tc_kernel", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, from "
                               "profiles/sandwich_tc_kernel_tfim32x32_m128.md (same kernel source)") if traffic else None,
            "peak_source": f"{src} bf16_tflops (burst: the kernel is timed per launch at full clock)",
            "flops_per_launch": k_fl / k_n if k_n else None, "avg_launch_ms": k_ms / k_n if k_n else None,
            "launches": k_n}
    line = {"metric": "H_eff matvecs/s at m=128", "value": value, "unit": "matvec/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "model": "tfim", "L": L, "h": H_FIELD, "m": M,
                       "n_de_placed": info["n_de"], "n_products_total": info["n_products"],
                       "node": info["node"], "node_counts_pairs01_02_12_triple_internal": list(counts),
                       "lanczos_depth": DEPTH, "algorithmic_flops_per_matvec": flops_mv,
                       "l2": "256 MB buffer written between timed steps; Lanczos basis 336 MB > L2",
                       "parallelism": f"replicas{world}"},
            "roofline": roof, "gpu_launches": int(launches), "e2e": e2e, "clocks": clk.summary(),
            "mixed_solve": solve, "fp32_krylov_basis": f32_basis}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(oracle_node_structure())
    if rank == 0 and world == 1 and not args.no_sweep:
        line["sweep"] = sweep_record(attn, torch)
    if rank == 0:
        print(json.dumps(line), flush=True)
    attn.attn_heff_destroy(H)
    attn.attn_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
