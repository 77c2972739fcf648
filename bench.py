#!/usr/bin/env python
"""Benchmark: encrypted 128x128 matrix products per second on one GB300.

One step = one batched pass of the hot path (he_hmatmul_batch) over B
products of 128x128 matrices encrypted at N = 2^16, level 20, modulus chain
60 + 20x40 bits, special primes 2x60 (the covariance configuration).
  value     batched products/s with ciphertexts resident in HBM
  plain     the same products one he_hmatmul call at a time (same GPU)
  e2e       the batched step through the C ABI from pinned host residues:
            upload + NTT, product, iNTT + download of every result
  roofline  live CUDA-event timing of the traced kernel classes (MultSum,
            forward / inverse NTT) over the timed region
  cpu_baseline / --impl reference: the CPU oracle on the host cores over a
            bounded sample (one Decompose, one MultSum, one ModDown at the
            same parameters), scaled by the per-product operation counts.

Multi-GPU (torchrun): every rank runs its own batch (independent products,
no collective on the data path); value = all ranks' products / max time.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HE 128×128 matmul/s batched vs plain, same GPU, bit-exact; keyswitch % HBM peak"
UNIT = "matmul/s"
N_MAT = 128
# DRAM bytes per algorithmic byte, from ncu captures of the same kernels
# (dram__bytes_read.sum + dram__bytes_write.sum of the launch over the bytes
# the traced class counts): the forward NTT's two passes each read and write
# the rows once, plus the row pass's twiddle misses (512-row captures of the
# two passes: 475.80 + 533.30 MB against 536.87 MB); MultSum reads the keys, the digits and c0 once and
# writes its outputs once (8 items x 4 hoisted rotations at level 20, the
# step's R^k / Z / T baby launches, compiled for 4 CTAs per SM: 2968.30 MB
# against 2982.15 MB).  Traffic grows with the rows / items of a launch, so
# per launch it is this ratio times the launch's algorithmic bytes.
TRAFFIC_RATIO = {"ntt_fwd": (475.80 + 533.30) / 536.87, "multsum": 2968.30 / 2982.15}
# baby-step count n1 used for each matrix dimension
N1_FOR = {16: 4, 32: 8, 64: 8, 128: 16}
LEVEL = 20
# per-product operation counts of the hoisted schedule at n=128, n1=16
# (Table 1 "Optimized" rows as the schedule performs them: Table 1 also counts
# the trivial j = 0 baby, the i = 0 giant and two chain steps, which the
# schedule does not perform)
OPS = {"MS": 564, "Dp": 178, "MD": 423}
# with one relinearisation per product instead of n = 128
OPS_ONCE = {"MS": 564 - 127, "Dp": 178 - 127, "MD": 423 - 127}


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.path = "/tmp/he_clocks_%d_%d.csv" % (os.getpid(), dev)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ multi-rank
def max_over_ranks(x, dist, device):
    """The slowest rank's time (every rank gets it); x itself without a group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, units_per_rank, seconds):
    """Whole-job throughput when every rank processes its own units (no data
    exchange): all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds


# -------------------------------------------------------------- cpu oracle
def oracle_sample(ops_per_step=1, ops=None):
    """Time the oracle's Decompose, MultSum and ModDown once each at logN 16,
    level 19 (the level of most key switches in the product) and scale by the
    per-product counts.  Returns (matmul/s, seconds spent, threads)."""
    import numpy as np

    from oracle.ckks import CKKS, Params
    t_all = time.time()
    P = Params(16, [60] + [40] * 20, [60, 60])
    he = CKKS(P, 77)
    he.gen_rotation_key(16)
    z = np.random.default_rng(1).uniform(-1, 1, P.S)
    ct = he.drop(he.encrypt_slots(z, P.L, obj=1), 19)
    t = {}
    for _ in range(ops_per_step):
        t0 = time.time()
        dg = he.modup(ct.c1, 19)
        t1 = time.time()
        u0, u1 = he.multsum(dg, he.rtk[P.galois(16)], 19)
        t2 = time.time()
        he.moddown2(u0, u1, 19)
        t3 = time.time()
        t.setdefault("Dp", []).append(t1 - t0)
        t.setdefault("MS", []).append(t2 - t1)
        t.setdefault("MD", []).append(t3 - t2)
    per = sum((ops or OPS)[k] * statistics.mean(v) for k, v in t.items())
    threads = env_int("OMP_NUM_THREADS", os.cpu_count() or 1)
    return 1.0 / per, time.time() - t_all, threads, {k: statistics.mean(v) for k, v in t.items()}


def oracle_full_product(logN, qbits, pbits, n, n1, sample_level):
    """The oracle on one whole encrypted n x n product (key generation
    excluded) next to the per-op extrapolation that cpu_baseline uses, at the
    same parameters: Decompose, MultSum and ModDown timed once each at
    `sample_level` and scaled by the product's own operation counts.  Returns
    a dict with both times and their ratio."""
    import numpy as np

    from oracle.ckks import CKKS, Params
    from oracle.hmm import HMM, matmul_rot_steps
    P = Params(logN, qbits, pbits)
    he = CKKS(P, 77)
    t0 = time.time()
    steps = matmul_rot_steps(n, n1, n1, P.S)
    for s in steps:
        he.gen_rotation_key(s)
    he.gen_relin_key()
    keygen = time.time() - t0
    rng = np.random.default_rng(2)
    z = [np.zeros(P.S), np.zeros(P.S)]
    for zz in z:
        zz[: n * n] = rng.uniform(-1, 1, n * n)
    a, b = he.encrypt_slots(z[0], P.L, obj=2), he.encrypt_slots(z[1], P.L, obj=3)
    he.cnt.reset()
    t0 = time.time()
    HMM(he).hmatmul(a, b, n, n1, n1)
    full = time.time() - t0
    cnt = {"MS": he.cnt.MS, "Dp": he.cnt.Dp, "MD": he.cnt.MD}
    ct = he.drop(a, sample_level)
    t0 = time.time()
    dg = he.modup(ct.c1, sample_level)
    t1 = time.time()
    u0, u1 = he.multsum(dg, he.rtk[P.galois(steps[0])], sample_level)
    t2 = time.time()
    he.moddown2(u0, u1, sample_level)
    t3 = time.time()
    per = {"Dp": t1 - t0, "MS": t2 - t1, "MD": t3 - t2}
    extra = sum(cnt[k] * per[k] for k in cnt)
    return {"workload": "%dx%d product, N=2^%d, %d q + %d p primes, level %d" % (n, n, logN, len(qbits), len(pbits),
                                                                             P.L),
            "measured_s": full, "extrapolated_s": extra, "ratio_measured_over_extrapolated": full / extra,
            "keygen_s": keygen, "counts": cnt, "per_op_s": per}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    if args.oracle_full:
        # the oracle on one whole 128x128 product at the bench's parameters
        # (minutes on the host cores), with the extrapolation beside it
        chk = oracle_full_product(16, [60] + [40] * 20, [60, 60], N_MAT, 16, 19)
        threads = env_int("OMP_NUM_THREADS", os.cpu_count() or 1)
        value = 1.0 / chk["measured_s"]
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1,
                "warmup": 0, "ms_per_step": 1000 * chk["measured_s"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": "one 128x128 encrypted matmul, N=2^16, q 60+20x40, p 2x60, level 20 "
                                       "(whole product, not extrapolated)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": "one whole product"},
                "extrapolation_check": chk,
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    vals = []
    for _ in range(args.warmup):
        oracle_sample()
    t0 = time.time()
    for _ in range(args.steps):
        v, _, threads, per = oracle_sample()
        vals.append(v)
    dt = time.time() - t0
    value = statistics.mean(vals)
    sample = ("per step: oracle Decompose + MultSum + ModDown once each at logN 16, level 19 (23 primes), "
              "scaled by the product's counts MS 564, Dp 178, MD 423 (an extrapolation: --oracle-full times one "
              "whole product)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "128x128 encrypted matmul, N=2^16, q 60+20x40, p 2x60, level 20"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours
def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import _lib, workloads

    local = env_int("LOCAL_RANK", 0)
    if args.preset == 1:     # N = 2^14, q 60+3x40, p 60: 32x32 products from the top level
        logN, level, n_mat, n1 = 14, 3, 32, 8
    else:
        logN, level, n_mat, n1 = 16, LEVEL, args.n, N1_FOR[args.n]
    Nn, S = 1 << logN, 1 << (logN - 1)
    torch.cuda.set_device(local)
    pk.build()
    L = _lib.lib()
    ctx = pk.he_ctx_create(pk.he_params_default(args.preset), 1000 + rank)
    if args.ms_variant is not None:
        pk.he_ctx_set_multsum_variant(ctx, args.ms_variant)
    if args.ntt_variant is not None:
        pk.he_ctx_set_ntt_variant(ctx, args.ntt_variant)
    # the library launches on this stream; every CUDA event below is recorded on it
    tstream = torch.cuda.Stream()
    pk.he_ctx_set_stream(ctx, tstream.cuda_stream)
    pk.he_keygen(ctx, pk.he_rot_steps_for_matmul(n_mat, n1, n1, S), True)
    B = args.batch
    mats = [workloads.matmul_pair(n_mat, 10 * (rank * 1000 + i)) for i in range(B)]
    cts = [(pk.he_encrypt_matrix(ctx, A, level, 2 * i), pk.he_encrypt_matrix(ctx, Bm, level, 2 * i + 1))
           for i, (A, Bm) in enumerate(mats)]
    once = bool(args.relin_once)
    jobs = [(a, b, n_mat, n1, n1, once) for a, b in cts]

    def batched_step():
        outs = pk.he_hmatmul_batch(jobs)
        for o in outs:
            pk.he_ct_free(o)

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (the first pass also fills the plaintext-diagonal cache)
    for _ in range(max(3, args.warmup)):
        batched_step()
    torch.cuda.synchronize()

    # correctness spot check of the benchmarked configuration (untimed)
    outs = pk.he_hmatmul_batch(jobs[:1])
    err = float(np.abs(pk.he_decrypt_matrix(ctx, outs[0], n_mat, n_mat) - mats[0][0] @ mats[0][1]).max())
    single_ref = pk.he_hmatmul(ctx, cts[0][0], cts[0][1], n_mat, n1, n1, relin_once=once)
    bitexact = bool(np.array_equal(pk.he_ct_export(ctx, single_ref), pk.he_ct_export(ctx, outs[0])))
    pk.he_ct_free(outs[0])

    # ---- timed region: K batched steps
    clocks = Clocks(local)
    pk.he_counters(ctx, reset=True)
    pk.he_trace_enable(ctx, True)
    for c in range(5):
        pk.he_trace_read(ctx, c, reset=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(tstream)
    torch.cuda.nvtx.range_push("timed")      # profilers select the timed launches by this range
    for _ in range(args.steps):
        batched_step()
    torch.cuda.nvtx.range_pop()
    e1.record(tstream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    tr = [pk.he_trace_read(ctx, c, reset=True) for c in range(5)]
    pk.he_trace_enable(ctx, False)
    launches = pk.he_counters(ctx, reset=True)["launches"]
    t_max = max_over_ranks(ms_total, dist, "cuda")
    value = weak_scaling_value(world, B * args.steps, t_max / 1000.0)

    # ---- plain: the same products one call at a time (untraced)
    ptimes = []
    for _ in range(max(1, args.plain_steps)):
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(tstream)
        for a, b in cts:
            o = pk.he_hmatmul(ctx, a, b, n_mat, n1, n1, relin_once=once)
            pk.he_ct_free(o)
        p1.record(tstream)
        torch.cuda.synchronize()
        ptimes.append(p0.elapsed_time(p1))
    plain = B / (statistics.median(ptimes) / 1000.0)

    # ---- the same batched step replayed as one captured CUDA graph
    graph = None
    if not args.no_graph:
        plan = pk.he_mm_plan_create(jobs)
        ginfo = pk.he_mm_plan_info(plan)
        for _ in range(3):
            for o in pk.he_mm_plan_run(plan):
                pk.he_ct_free(o)
        outs_g = pk.he_mm_plan_run(plan)
        gbit = bool(np.array_equal(pk.he_ct_export(ctx, outs_g[0]), pk.he_ct_export(ctx, single_ref)))
        for o in outs_g:
            pk.he_ct_free(o)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(tstream)
        for _ in range(args.steps):
            for o in pk.he_mm_plan_run(plan):
                pk.he_ct_free(o)
        g1.record(tstream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1)
        graph = {"value": B * args.steps / (gms / 1000.0), "unit": UNIT, "ms_per_step": gms / args.steps,
                 "launches_per_step": ginfo["launches"], "plan_bytes": ginfo["bytes"],
                 "bitexact_vs_batch": gbit}
        pk.he_mm_plan_destroy(plan)
    pk.he_ct_free(single_ref)

    # ---- the same products with one relinearisation each (not the paper's
    #      DMatrixMult: n - 1 fewer key switches per product)
    once_line = None
    if not once and not args.no_once:
        jobs1 = [(a, b, n_mat, n1, n1, True) for a, b in cts]
        for _ in range(2):
            for o in pk.he_hmatmul_batch(jobs1):
                pk.he_ct_free(o)
        o1 = pk.he_hmatmul_batch(jobs1[:1])
        s1 = pk.he_hmatmul(ctx, cts[0][0], cts[0][1], n_mat, n1, n1, relin_once=True)
        ob = bool(np.array_equal(pk.he_ct_export(ctx, o1[0]), pk.he_ct_export(ctx, s1)))
        oerr = float(np.abs(pk.he_decrypt_matrix(ctx, o1[0], n_mat, n_mat) - mats[0][0] @ mats[0][1]).max())
        pk.he_ct_free(o1[0])
        pk.he_ct_free(s1)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(tstream)
        for _ in range(args.steps):
            for o in pk.he_hmatmul_batch(jobs1):
                pk.he_ct_free(o)
        r1.record(tstream)
        torch.cuda.synchronize()
        rms = r0.elapsed_time(r1)
        once_line = {"value": B * args.steps / (rms / 1000.0), "unit": UNIT, "ms_per_step": rms / args.steps,
                     "batch_equals_single_bitexact": ob, "max_abs_err": oerr,
                     "note": "relin_once=1: the n tensors summed, one key switch per product (not DMatrixMult)"}

    # ---- e2e through the C ABI from pinned host memory
    w_in = 2 * (level + 1) * Nn
    w_out = 2 * (level - 3 + 1) * Nn
    host_in = torch.empty((B, 2, w_in), dtype=torch.int64, pin_memory=True)
    host_out = torch.empty((B, w_out), dtype=torch.int64, pin_memory=True)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    for i, (a, b) in enumerate(cts):
        host_in[i, 0].numpy()[:] = pk.he_ct_export(ctx, a).view(np.int64).ravel()
        host_in[i, 1].numpy()[:] = pk.he_ct_export(ctx, b).view(np.int64).ravel()
    scale = pk.he_ct_info(cts[0][0])[1]

    def e2e_step():
        hs = []
        for i in range(B):
            for j in range(2):
                h = ctypes.c_void_p()
                ptr = ctypes.cast(host_in[i, j].data_ptr(), u64p)
                _lib.check(L.he_ct_import(ctx, ptr, level, scale, S, ctypes.byref(h)))
                hs.append(h)
        outs = pk.he_hmatmul_batch([(hs[2 * i], hs[2 * i + 1], n_mat, n1, n1, once) for i in range(B)])
        for i, o in enumerate(outs):
            _lib.check(L.he_ct_export(o, ctypes.cast(host_out[i].data_ptr(), u64p)))
            pk.he_ct_free(o)
        for h in hs:
            pk.he_ct_free(h)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_val = weak_scaling_value(world, B * max(1, args.e2e_steps), e2e_dt)

    # ---- rooflines
    pk_ = peaks()
    hbm = pk_.get("hbm_gbs")
    hbm_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    bfly_peak = pk.he_bench_butterfly(4000)
    mac_peak = pk.he_bench_mac(4000)

    def hbm_roof(t):
        if not t["count"]:
            return None
        avg_s = t["ms"] / t["count"] / 1000.0
        ach = t["bytes"] / t["count"] / avg_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_source": hbm_src,
                "traffic": (TRAFFIC_RATIO["multsum"] * t["bytes"] / t["count"]
                            if args.preset == 2 and TRAFFIC_RATIO["multsum"] else None),
                "launches": t["count"], "avg_us": avg_s * 1e6,
                "alu": mac_roof(t)}

    def mac_roof(t):
        # the second ceiling of MultSum: its digit-key products against the
        # measured rate of the 96-bit product accumulation
        if not t["count"] or not t.get("ops"):
            return None
        rate = t["ops"] / (t["ms"] / 1e3) / 1e9
        return {"achieved": rate, "peak": mac_peak / 1e9, "unit": "G products/s", "frac": rate / (mac_peak / 1e9),
                "peak_source": "measured 96-bit product-accumulate microbenchmark on this GPU"}

    def ntt_roof(t, ratio=None):
        if not t["count"]:
            return None
        avg_s = t["ms"] / t["count"] / 1000.0
        words = t["bytes"] / t["count"] / 16.0                     # rows * N per launch
        bfly = words / 2.0 * logN                                   # (N/2) log2 N per row
        ach = bfly / avg_s / 1e9
        peak = bfly_peak / 1e9
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gbutterfly/s", "frac": ach / peak,
                "peak_source": "measured lazy-Shoup butterfly microbenchmark on this GPU",
                "traffic": ratio * t["bytes"] / t["count"] if ratio else None,
                "launches": t["count"], "avg_us": avg_s * 1e6,
                "hbm_gbs": t["bytes"] / t["count"] / avg_s / 1e9}

    roof_ms = hbm_roof(tr[0])
    roof_nf = ntt_roof(tr[1], TRAFFIC_RATIO["ntt_fwd"] if args.preset == 2 else None)
    roof_ni = ntt_roof(tr[2])
    totals = {"multsum": tr[0]["ms"], "ntt_fwd": tr[1]["ms"], "ntt_inv": tr[2]["ms"]}
    dominant = max(totals, key=totals.get)
    # the two basis conversions (integer ALU with streaming stores): time and
    # algorithmic GB/s, for attribution
    conv = {name: {"ms": t["ms"], "launches": t["count"],
                   "algorithmic_gbs": t["bytes"] / (t["ms"] / 1e3) / 1e9 if t["ms"] else None}
            for name, t in (("modup_bconv", tr[3]), ("moddown_bconv", tr[4]))}
    roof = {"multsum": roof_ms, "ntt_fwd": roof_nf, "ntt_inv": roof_ni}[dominant]
    roof = dict(roof, kernel=dominant, share_of_step=totals[dominant] / ms_total)

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu and args.preset == 2 and n_mat == N_MAT:
        ops = OPS_ONCE if once else OPS
        v, spent, threads, per = oracle_sample(ops=ops)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "extrapolated: oracle Decompose + MultSum + ModDown once each at logN 16, level 19, 23 "
                         "primes (%.1f s incl. key generation), scaled by the product's counts MS %d, Dp %d, MD %d"
                         % (spent, ops["MS"], ops["Dp"], ops["MD"]),
               "per_op_s": per}
        if not once:
            # the same extrapolation checked against a whole product where
            # the oracle finishes one in seconds (config 1: 32x32, N = 2^14)
            cpu["extrapolation_check_m1"] = oracle_full_product(14, [60, 40, 40, 40], [60], 32, 8, 2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batch of %d encrypted %dx%d matmuls, N=2^%d, %s, level %d, n1_z=n1_t=%d, %s"
                               % (B, n_mat, n_mat, logN, "q 60+20x40, p 2x60" if args.preset == 2 else
                                  "q 60+3x40, p 60", level, n1,
                                  "one relinearisation per product" if once else
                                  "relinearised per A^(k)B^(k) term (DMatrixMult)"),
                   "relin_once": once,
                   "batch_per_gpu": B, "n": n_mat, "logN": logN, "level": level,
                   "l2": ("inputs larger than L2 (rotation keys and %d ciphertext pairs streamed per step)" % B
                          if args.preset == 2 else "no flush: keys and ciphertexts fit in L2 (small-ring case)"),
                   "parallelism": "replicas" if world == 1 else "independent products per rank"},
        "plain": {"value": plain, "unit": UNIT, "note": "same products, one he_hmatmul call each"},
        "batched_over_plain": value / world / plain,
        "roofline": roof, "roofline_keyswitch": roof_ms, "roofline_ntt_fwd": roof_nf, "roofline_ntt_inv": roof_ni,
        "kernel_time_ms": dict(totals, modup_bconv=tr[3]["ms"], moddown_bconv=tr[4]["ms"]),
        "conversions": conv,
        "graph": graph,
        "relin_once": once_line,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": B * 2 * w_in * 8,
                "d2h_bytes_per_step": B * w_out * 8},
        "clocks": ck, "gpu_launches": launches,
        "check": {"max_abs_err": err, "tol": 1e-4, "batch_equals_single_bitexact": bitexact},
        "ntt_launch_tuning": [x for x in pk.he_autotune_log(ctx).splitlines() if x.startswith("ntt")],
        "multsum_launch_picks": multsum_picks(pk.he_autotune_log(ctx)),
    }
    if n_mat != N_MAT:
        line["note"] = "profiling case (n=%d), not the benchmark workload" % n_mat
    print(json.dumps(line), flush=True)
    pk.he_ctx_destroy(ctx)


def multsum_picks(log):
    """The MultSum launch plan the tuner kept for each (level, items, rotations):
    the fastest of its timed candidates (log lines "multsum level L B b G g
    chunk c BI v stream s ms t"; BI above 100 names launch variant BI - 100)."""
    best = {}
    for ln in log.splitlines():
        f = ln.split()
        if len(f) != 15 or f[0] != "multsum":
            continue
        key = (int(f[2]), int(f[4]), int(f[6]))
        t = float(f[14])
        if key not in best or t < best[key][0]:
            best[key] = (t, int(f[8]), int(f[10]), int(f[12]))
    picks = ["level %d B %d G %d: %d keys per launch, %s, %.4f ms" %
             (k + (v[1], ("variant %d" % (v[2] - 100)) if v[2] > 100 else "%d items per CTA%s" %
                   (v[2], ", streaming" if v[3] else ""), v[0]))
             for k, v in sorted(best.items())]
    # the fused C^k babies: "multsum_ck level L B b G g chunk c BI v ms t"
    # (BI 0: rotations split over the warps)
    ck = {}
    for ln in log.splitlines():
        f = ln.split()
        if len(f) != 13 or f[0] != "multsum_ck":
            continue
        key = (int(f[2]), int(f[4]), int(f[6]))
        t = float(f[12])
        if key not in ck or t < ck[key][0]:
            ck[key] = (t, int(f[8]), int(f[10]))
    picks += ["C^k fused, level %d B %d G %d: %d keys per launch, %s, %.4f ms" %
              (k + (v[1], "rotations split over the warps" if v[2] == 0 else "%d items per CTA" % v[2], v[0]))
              for k, v in sorted(ck.items())]
    return picks


def _cov_keys(pk, ctx, n, n1, S, dcd=0):
    """Rotation keys of HCovMtrx with n x n blocks: the block products (with
    the decomposition at maximum diagonal dcd if given), transpositions,
    Aggregate sums and replication; and the relinearisation key."""
    steps = set(pk.he_rot_steps_for_matmul(n, n1, n1, S)) | set(pk.he_rot_steps_for_transpose(n, n1, S))
    if dcd:
        steps |= set(pk.he_rot_steps_for_sched(n, n1, n1, S, dcd, dcd))
    i = 1
    while i < n * n:
        steps |= {i % (n * n), (-i) % (n * n)}
        i <<= 1
    steps.discard(0)
    pk.he_keygen(ctx, sorted(steps), True)


def run_covariance(args):
    """Config 2: encrypted covariance of a 256x256 low-rank dataset (128x128
    blocks, N=2^16), with undecomposed block products and with the Diagonal
    Convergence Decomposition at maximum diagonal 32 (the covariance setting
    of Sec. 7)."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import workloads
    pk.build()
    n, n1, s, t = 128, 16, args.rows, 256
    ctx = pk.he_ctx_create(pk.he_params_default(2), 42)
    _cov_keys(pk, ctx, n, n1, 1 << 15)
    X = workloads.lowrank_dataset(s, t, 2)
    nrb = -(-s // n)
    Xp = np.zeros((nrb * n, t))
    Xp[:s] = X
    blocks = [pk.he_encrypt_matrix(ctx, Xp[l * n:(l + 1) * n, j * n:(j + 1) * n], 20, 100 + l * 2 + j)
              for l in range(nrb) for j in range(2)]
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / s

    def run(dcd):
        C = pk.he_covariance(ctx, blocks, nrb, 2, n, s, False, n1, n1, dcd_z=dcd, dcd_t=dcd)   # warm-up
        for h in C:
            pk.he_ct_free(h)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            C = pk.he_covariance(ctx, blocks, nrb, 2, n, s, False, n1, n1, dcd_z=dcd, dcd_t=dcd)
            times.append(time.perf_counter() - t0)
            Cd = [pk.he_decrypt_matrix(ctx, h, n, n) for h in C]
            lv = pk.he_ct_info(C[0])[0]
            for h in C:
                pk.he_ct_free(h)
        err = max(float(np.abs(Cd[a * 2 + b] - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max())
                  for a in range(2) for b in range(2))
        return statistics.median(times) * 1000, err, lv

    ms, err, lv = run(0)
    ms32, err32, lv32 = run(32)
    # rotation keys the block products need (Table 2): undecomposed and at n' = 32
    S = 1 << 15
    keys0 = len(pk.he_rot_steps_for_sched(n, n1, n1, S, 0, 0))
    keys32 = len(pk.he_rot_steps_for_sched(n, n1, n1, S, 32, 32))
    print(json.dumps({"metric": "encrypted covariance time (HCovMtrx)", "value": ms, "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
                      "config": {"workload": "covariance of a %dx256 low-rank dataset, 128x128 blocks, N=2^16, "
                                             "q 60+20x40, p 2x60" % s, "matmuls": 3 * nrb},
                      "end_level": lv, "product_rotation_keys": keys0,
                      "decomposed_n32": {"value": ms32, "unit": "ms", "end_level": lv32,
                                         "product_rotation_keys": keys32, "max_abs_err_vs_fp64": err32},
                      "check": {"max_abs_err_vs_fp64": err, "tol": 1e-4}}), flush=True)
    pk.he_ctx_destroy(ctx)


def run_pca(args):
    """Config 3: top-8 eigenvectors by HPowerMethod + HEigenShift on the
    encrypted 256x256 covariance, chain 60 + 13x40, p 2x60 (Sec. 7.2.3)."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import workloads
    pk.build()
    n, n1, s, t, k = 128, 16, 256, 256, 2
    l_E, l_P = args.components, args.pm_iters
    # covariance in the covariance context (config 2)
    ctx2 = pk.he_ctx_create(pk.he_params_default(2), 42)
    _cov_keys(pk, ctx2, n, n1, 1 << 15)
    X = workloads.lowrank_dataset(s, t, 2)
    blocks = [pk.he_encrypt_matrix(ctx2, X[l * n:(l + 1) * n, j * n:(j + 1) * n], 20, 100 + l * 2 + j)
              for l in range(2) for j in range(2)]
    t0 = time.perf_counter()
    C2 = pk.he_covariance(ctx2, blocks, 2, k, n, s, False, n1, n1)
    cov_s = time.perf_counter() - t0
    # interactive refresh into the PowerMethod context, with the public
    # pre-scale by the feature count d = 256 (norm bound B = b^2 c d, b = 1)
    ctx3 = _pm_context(pk, n, 1 << 15)
    C3 = []
    for a in range(k):
        for b in range(k):
            blk = pk.he_decrypt_matrix(ctx2, C2[a * k + b], n, n) * t
            C3.append(pk.he_replicate(ctx3, pk.he_encrypt_matrix(ctx3, blk, 13, 200 + a * k + b), n))
    rng = np.random.default_rng(3)
    v0s = []
    for m in range(l_E):
        v0 = rng.standard_normal(t)
        v0 /= np.linalg.norm(v0)
        for j in range(k):
            v0s.append(pk.he_replicate(ctx3, pk.he_encrypt_matrix(ctx3, np.tile(v0[j * n:(j + 1) * n], (n, 1)), 13,
                                                                  300 + m * k + j), n))
    counts = pk.he_lazy_normalization_schedule(l_P)
    Xc = X - X.mean(0)
    w, U = np.linalg.eigh(Xc.T @ Xc / s)
    w, U = w[::-1], U[:, ::-1]

    def run(compose, pack=False):
        """he_pca on the same inputs; wall time, refreshes and accuracy."""
        pk.he_ctx_set_newton_composition(ctx3, compose)
        pk.he_ctx_set_packed_refresh(ctx3, pack)
        rs = pk.he_refresh_state(1 << 20, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lams, Vs, axes = pk.he_pca(ctx3, C3, k, n, l_E, v0s, 0, l_P, counts, 2.0 ** 16, rs)
        pm_s = time.perf_counter() - t0
        cos, lam_he, vecs = [], [], []
        for m in range(l_E):
            parts = []
            for j in range(k):
                d = pk.he_decrypt_matrix(ctx3, Vs[m][j], n, n)
                parts.append(d[0] if axes[m] == 0 else d[:, 0])
            v = np.concatenate(parts)
            vecs.append(v)
            cos.append(float(abs(v @ U[:, m]) / np.linalg.norm(v)))
            lam_he.append(float(pk.he_decrypt_slots(ctx3, lams[m], 1)[0] / t))
        Vm = np.array([v / np.linalg.norm(v) * np.sign(v @ U[:, m]) for m, v in enumerate(vecs)])
        Ut = U[:, :l_E].T
        r2v = 1 - ((Vm - Ut) ** 2).sum() / ((Ut - Ut.mean()) ** 2).sum()
        for h in lams + [x for V in Vs for x in V]:
            pk.he_ct_free(h)
        # agreement with the FP64 run of the same schedule: the CKKS error alone
        run.vs_fp64 = [float(abs(v @ f) / (np.linalg.norm(v) * np.linalg.norm(f))) for v, f in zip(vecs, f_vec)]
        return pm_s, rs.count, cos, lam_he, float(r2v)

    # The same method in FP64 on the exact covariance (pre-scaled by d like
    # the encrypted one): the same start vectors, PowerMethod iterations,
    # TaylorInit + Newton counts of Lazy Normalization (Sec. 6.1.2) and
    # EigenShift deflation (Sec. 6.2).  Its cosines against eigh are the
    # method's own convergence; the encrypted run adds the CKKS error.
    def fp64_same_schedule():
        Cs = (Xc.T @ Xc / s) * t
        x0 = 2.0 ** 15 + 1.0
        rs_ = np.random.default_rng(3)
        out_cos, out_lam, out_vec = [], [], []
        for m in range(l_E):
            v = rs_.standard_normal(t)
            v /= np.linalg.norm(v)
            for it in range(l_P):
                yv = Cs @ v
                x = yv @ yv
                inv = x0 ** -0.5 * (1.5 - x / (2.0 * x0))
                for _ in range(counts[it]):
                    inv = 0.5 * inv * (3.0 - x * inv * inv)
                v = yv * inv
            lam = (Cs @ v) @ v
            out_cos.append(float(abs(v @ U[:, m]) / np.linalg.norm(v)))
            out_lam.append(float(lam / t))
            out_vec.append(v)
            Cs = Cs - lam * np.outer(v, v)
        return out_cos, out_lam, out_vec

    f_cos, f_lam, f_vec = fp64_same_schedule()
    pm_s, refreshes, cos, lam_he, r2v = run(False)
    run_vs_fp64 = run.vs_fp64
    comp = packed = None
    if not args.no_compose:
        c_s, c_ref, c_cos, c_lam, c_r2 = run(True)
        comp = {"value": c_s, "unit": "s", "refreshes": c_ref, "cosine_vs_eigh": c_cos, "lambda_he": c_lam,
                "R2_V": c_r2, "note": "pairs of Newton steps as five-level composites (Sec. 7)"}
        p_s, p_ref, p_cos, p_lam, p_r2 = run(True, True)
        packed = {"value": p_s, "unit": "s", "refreshes": p_ref, "cosine_vs_eigh": p_cos, "lambda_he": p_lam,
                  "R2_V": p_r2, "note": "composite Newton steps and the packed eigenvector refresh (App. C)"}
    print(json.dumps({"metric": "encrypted PCA time (HPowerMethod + HEigenShift, top-%d)" % l_E, "value": pm_s,
                      "unit": "s", "higher_is_better": False, "n_gpus": 1,
                      "config": {"workload": "top-%d eigenvectors of the encrypted covariance of a 256x256 low-rank "
                                             "dataset; PowerMethod at N=2^16, q 60+13x40, p 2x60; l_P=%d; Newton "
                                             "counts %s; covariance pre-scaled by d=256" % (l_E, l_P, counts)},
                      "covariance_s": cov_s, "refreshes": refreshes, "cosine_vs_eigh": cos,
                      "lambda_he": lam_he, "lambda_fp64": [float(x) for x in w[:l_E]], "R2_V": r2v,
                      "fp64_same_schedule": {"cosine_vs_eigh": f_cos, "lambda": f_lam,
                                             "note": "the PowerMethod of the encrypted run (same start vectors, "
                                                     "l_P, Newton counts, deflation) in FP64 on the exact "
                                                     "covariance"},
                      "cosine_he_vs_fp64_same_schedule": run_vs_fp64,
                      "eigen_gaps": [float(w[m + 1] / w[m]) for m in range(l_E)],
                      "per_pm_iteration_s": pm_s / (l_E * (l_P + 1)), "composed_newton": comp,
                      "composed_newton_packed_refresh": packed}), flush=True)
    pk.he_ctx_destroy(ctx3)
    pk.he_ctx_destroy(ctx2)



def _pm_context(pk, n, S):
    """The PowerMethod context (chain 60 + 13x40, p 2x60) with the rotation
    keys of Aggregate-style sums (+-2^i) and of replication."""
    ctx3 = pk.he_ctx_create(pk.he_params_default(3), 43)
    steps = set()
    i = 1
    while i < n * n:
        steps |= {i % (n * n), (-i) % (n * n)}
        i <<= 1
    r = n * n
    while r < S:
        steps.add((-r) % S)
        r *= 2
    steps.discard(0)
    pk.he_keygen(ctx3, sorted(steps), True)
    return ctx3


def run_served(args):
    """Config 5: Poisson arrivals of X^T X row-block jobs (one 128-row block of
    a 256-feature stream each, accumulated into one encrypted X^T X / s),
    128x128 products, 256x256 covariances and top-k PCA jobs, served by
    he_server over resident keys: one worker per context (covariance chain at
    N=2^16 and the PowerMethod chain), products of all queued jobs merged into
    batched passes, admission against a device-memory budget."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import workloads
    pk.build()
    n, n1, k, t = 128, 16, 2, 256
    if args.served_rows:
        # the streamed dataset: served_rows x 256 as ceil(rows / 128) row blocks
        blocks_total = -(-args.served_rows // n)
        mix = workloads.served_job_mix(args.rate, args.duration, 5, workloads.SERVED_STREAM_WEIGHTS, blocks_total)
        s_rows = args.served_rows
    else:
        mix = workloads.served_job_mix(args.rate, args.duration, 5)
        s_rows = None
    ctx2 = pk.he_ctx_create(pk.he_params_default(2), 52)
    _cov_keys(pk, ctx2, n, n1, 1 << 15, args.served_dcd)
    # the covariance jobs' block products: decomposed at maximum diagonal
    # served_dcd (Sec. 7 runs the covariance with n' = 32), or undecomposed
    dk = dict(dcd_z=args.served_dcd, dcd_t=args.served_dcd)
    # client side, before the timed region: encrypt every input
    n_blk = max(1, sum(1 for _, kd in mix if kd == "xtx_block"))
    if s_rows:
        # every arriving block of the dataset; the total row count s is the
        # dataset's (the accumulator divides by it), the last block zero-padded
        Xfull = workloads.lowrank_dataset(s_rows, t, 6)
        Xs = np.zeros((n * max(n_blk, -(-s_rows // n)), t))
        Xs[:s_rows] = Xfull
    else:
        s_rows = n * n_blk
        Xs = workloads.lowrank_dataset(n * n_blk, t, 6)
    stream = [[pk.he_encrypt_matrix(ctx2, Xs[l * n:(l + 1) * n, j * n:(j + 1) * n], 20, 10000 + 2 * l + j)
               for j in range(k)] for l in range(n_blk)]
    pairs = [workloads.matmul_pair(n, 70 + i) for i in range(4)]
    mm = [(pk.he_encrypt_matrix(ctx2, A, 20, 500 + 2 * i), pk.he_encrypt_matrix(ctx2, B, 20, 501 + 2 * i))
          for i, (A, B) in enumerate(pairs)]
    Xc2 = workloads.lowrank_dataset(256, t, 2)
    cov_in = [pk.he_encrypt_matrix(ctx2, Xc2[l * n:(l + 1) * n, j * n:(j + 1) * n], 20, 600 + 2 * l + j)
              for l in range(2) for j in range(k)]
    big_rows = 4096
    want_big = any(kd == "covariance_large" for _, kd in mix)
    Xbig = workloads.lowrank_dataset(big_rows, t, 7) if want_big else None
    cov_big = ([pk.he_encrypt_matrix(ctx2, Xbig[l * n:(l + 1) * n, j * n:(j + 1) * n], 20, 20000 + 2 * l + j)
                for l in range(big_rows // n) for j in range(k)] if want_big else [])
    want_pca = any(kd == "pca" for _, kd in mix) and not args.no_pca
    ctxs = [ctx2]
    pca_in, counts = [], None
    if want_pca:
        ctx3 = _pm_context(pk, n, 1 << 15)
        ctxs.append(ctx3)
        Xc = Xc2 - Xc2.mean(0)
        Cs = Xc.T @ Xc / 256 * t
        pca_in = [pk.he_replicate(ctx3, pk.he_encrypt_matrix(ctx3, Cs[a * n:(a + 1) * n, b * n:(b + 1) * n], 13,
                                                             700 + a * k + b), n) for a in range(k) for b in range(k)]
        rng = np.random.default_rng(3)
        for m in range(args.components):
            v0 = rng.standard_normal(t)
            v0 /= np.linalg.norm(v0)
            pca_in += [pk.he_replicate(ctx3, pk.he_encrypt_matrix(ctx3, np.tile(v0[j * n:(j + 1) * n], (n, 1)), 13,
                                                                  800 + m * k + j), n) for j in range(k)]
        counts = pk.he_lazy_normalization_schedule(args.pm_iters)
    srv = pk.he_server_create(ctxs, args.budget_gb * 1e9, args.max_batch)

    def submit(kind, idx, acc_id=1):
        if kind == "xtx_block":
            return pk.he_server_submit(srv, pk.HE_JOB_XTX_BLOCK, stream[idx], n=n, n1z=n1, n1t=n1, k=k,
                                       s=s_rows, acc_id=acc_id, **dk)
        if kind == "matmul":
            a, b = mm[idx % len(mm)]
            return pk.he_server_submit(srv, pk.HE_JOB_MATMUL, [a, b], n=n, n1z=n1, n1t=n1)
        if kind == "covariance":
            return pk.he_server_submit(srv, pk.HE_JOB_COVARIANCE, cov_in, n=n, n1z=n1, n1t=n1, n_row_blocks=2, k=k,
                                       s=256, **dk)
        if kind == "covariance_large":
            return pk.he_server_submit(srv, pk.HE_JOB_COVARIANCE, cov_big, n=n, n1z=n1, n1t=n1,
                                       n_row_blocks=big_rows // n, k=k, s=big_rows, **dk)
        return pk.he_server_submit(srv, pk.HE_JOB_PCA, pca_in, n=n, k=k, l_E=args.components, l_P=args.pm_iters,
                                   axis=0, counts=counts, B2=2.0 ** 16, refresh_obj=(1 << 20) + (idx << 16))

    def drain(ids):
        outs = {}
        for j, kind in ids:
            pk.he_server_wait(srv, j, 3600.0)
            try:
                outs[j] = (kind, pk.he_server_result(srv, j)[0])
            except pk.HeError as e:
                outs[j] = (kind, e)
        return outs

    # warm-up (plaintext-diagonal caches of every shape and level), untimed
    warm = [(submit("matmul", 0), "matmul"), (submit("covariance", 0), "covariance"),
            (submit("xtx_block", 0, acc_id=0), "xtx_block")]
    warm.append((pk.he_server_submit(srv, pk.HE_JOB_XTX_FINAL, [], ctx=ctx2, n=n, n1z=n1, n1t=n1, k=k, acc_id=0,
                                     **dk), "final"))
    for kind, res in drain(warm).values():
        if not isinstance(res, Exception):
            for h in res:
                pk.he_ct_free(h)
    pk.he_server_destroy(srv)                 # a fresh server for the timed run (statistics from zero)
    srv = pk.he_server_create(ctxs, args.budget_gb * 1e9, args.max_batch)
    torch.cuda.synchronize()
    # ---- timed: arrivals in real time
    ids, nb, counters = [], 0, {}
    clocks = Clocks(0)
    clocks.start()
    t0 = time.perf_counter()
    for at, kind in mix:
        dt = t0 + at - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        idx = counters.get(kind, 0)
        counters[kind] = idx + 1
        try:
            ids.append((submit(kind, nb if kind == "xtx_block" else idx), kind))
            nb += kind == "xtx_block"
        except pk.HeError as e:
            if e.code != pk.HE_ERR_ADMISSION:     # counted by the server's statistics
                raise
    fin = pk.he_server_submit(srv, pk.HE_JOB_XTX_FINAL, [], ctx=ctx2, n=n, n1z=n1, n1t=n1, k=k, acc_id=1, **dk)
    ids.append((fin, "final"))
    res = drain(ids)
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    names = {1: "matmul", 2: "covariance (both sizes)", 3: "xtx_block", 4: "xtx_final", 5: "pca"}
    per_kind = {}
    for kd, name in names.items():
        st = pk.he_server_stats(srv, kd)
        if st["submitted"]:
            per_kind[name] = {x: st[x] for x in ("submitted", "admitted", "waited", "rejected", "completed",
                                                 "failed", "p50_ms", "p99_ms", "mean_ms", "max_ms")}
    st = pk.he_server_stats(srv, 0)
    pk.he_server_destroy(srv)
    # ---- checks against FP64 (decrypted, untimed)
    check = {}
    xtx = res[fin][1]
    if not isinstance(xtx, Exception):
        Xb = Xs[:n * nb]
        ref = Xb.T @ Xb / s_rows
        check["xtx_max_abs_err"] = max(float(np.abs(pk.he_decrypt_matrix(ctx2, xtx[a * k + b], n, n) -
                                                    ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max())
                                       for a in range(k) for b in range(k))
    for j, (kind, r) in res.items():
        if isinstance(r, Exception):
            continue
        if kind == "matmul" and "matmul_max_abs_err" not in check:
            A, B = pairs[[jj for jj, kk in ids if kk == "matmul"].index(j) % len(mm)]
            check["matmul_max_abs_err"] = float(np.abs(pk.he_decrypt_matrix(ctx2, r[0], n, n) - A @ B).max())
        if kind == "covariance_large" and "covariance_large_max_abs_err" not in check:
            Xc = Xbig - Xbig.mean(0)
            ref = Xc.T @ Xc / big_rows
            check["covariance_large_max_abs_err"] = max(
                float(np.abs(pk.he_decrypt_matrix(ctx2, r[a * k + b], n, n) - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max())
                for a in range(k) for b in range(k))
        if kind == "covariance" and "covariance_max_abs_err" not in check:
            Xc = Xc2 - Xc2.mean(0)
            ref = Xc.T @ Xc / 256
            check["covariance_max_abs_err"] = max(
                float(np.abs(pk.he_decrypt_matrix(ctx2, r[a * k + b], n, n) - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max())
                for a in range(k) for b in range(k))
        for h in r:
            pk.he_ct_free(h)
    failed = sum(1 for _, r in res.values() if isinstance(r, Exception))
    print(json.dumps({
        "metric": "served encrypted jobs/s (Poisson arrivals; continuous batching over resident keys)",
        "value": st["jobs_per_s"], "unit": "jobs/s", "higher_is_better": True, "n_gpus": 1,
        "latency_ms": {"p50": st["p50_ms"], "p99": st["p99_ms"], "mean": st["mean_ms"], "max": st["max_ms"]},
        "per_kind": per_kind,
        "admitted": st["admitted"], "waited": st["waited"], "rejected": st["rejected"], "failed": failed,
        "ticks": st["ticks"], "products": st["products"],
        "products_per_tick": st["products"] / max(1, st["ticks"]), "max_products_per_tick": st["max_products_per_tick"],
        "key_bytes": st["key_bytes"], "wall_s": wall, "clocks": ck,
        # the arrival rate against what the server completes: when it cannot
        # keep up, the queue grows and drains after the last arrival
        "backlog": {"arrivals_per_s": len(mix) / args.duration, "completed_per_s": st["jobs_per_s"],
                    "keeps_up": st["jobs_per_s"] >= len(mix) / args.duration,
                    "drain_s_after_last_arrival": wall - (mix[-1][0] if mix else 0.0)},
        "config": {"workload": "Poisson arrivals at %.2f jobs/s for %.0f s: X^T X row blocks of a %dx256 dataset "
                               "(128x256 each, one accumulator, %d of %d blocks arrived), 256x256 and 4096x256 "
                               "covariances, top-%d PCA%s; N=2^16, covariance chain 60+20x40 / PowerMethod chain "
                               "60+13x40, p 2x60"
                               % (args.rate, args.duration, s_rows, nb, -(-s_rows // n), args.components,
                                  "" if args.served_rows else ", 128x128 products"),
                   "budget_gb": args.budget_gb, "max_batch": args.max_batch, "jobs": len(mix),
                   "covariance_products": "decomposed, n' = %d (Sec. 7)" % args.served_dcd if args.served_dcd
                   else "undecomposed"},
        "check": dict(check, tol=1e-4)}), flush=True)
    for h in [x for blk in stream for x in blk] + [x for p in mm for x in p] + cov_in + cov_big + pca_in:
        pk.he_ct_free(h)
    for c in ctxs:
        pk.he_ctx_destroy(c)


def run_keyswitch(args):
    """Hoisted key-switched rotations alone (he_rotate_hoisted): B ciphertexts
    at level 20 of the 60 + 20x40 / 2x60 chain (N = 2^16), each Decomposed
    once and rotated by R steps; every MultSum launch reads one rotation key
    for all B ciphertexts.  Device time of the traced kernel classes; the
    MultSum roofline is the key switch's HBM roofline."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(2), 11)
    if args.ms_variant is not None:
        pk.he_ctx_set_multsum_variant(ctx, args.ms_variant)
    if args.ntt_variant is not None:
        pk.he_ctx_set_ntt_variant(ctx, args.ntt_variant)
    if args.ntt_chunk is not None:
        pk.he_ctx_set_ntt_chunk(ctx, args.ntt_chunk)
    tstream = torch.cuda.Stream()
    pk.he_ctx_set_stream(ctx, tstream.cuda_stream)
    R, B = args.rot_steps, args.batch
    steps = [1 + 37 * i for i in range(R)]
    pk.he_keygen(ctx, steps, False)
    rng = np.random.default_rng(13)
    cts = [pk.he_encrypt_slots(ctx, rng.uniform(-1, 1, 1 << 15), LEVEL, 7000 + i) for i in range(B)]

    def step():
        for row in pk.he_rotate_hoisted(ctx, cts, steps):
            for h in row:
                pk.he_ct_free(h)

    for _ in range(max(3, args.warmup)):
        step()
    pk.he_trace_enable(ctx, True)
    for c in range(5):
        pk.he_trace_read(ctx, c, reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(tstream)
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        step()
    torch.cuda.nvtx.range_pop()
    e1.record(tstream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tr = [pk.he_trace_read(ctx, c, reset=True) for c in range(5)]
    pk.he_trace_enable(ctx, False)
    hbm = peaks().get("hbm_gbs") or 6800.0
    mac_peak = pk.he_bench_mac(4000) / 1e9
    t = tr[0]
    avg = t["ms"] / t["count"] / 1e3
    ach = t["bytes"] / t["count"] / avg / 1e9
    prod = t["ops"] / (t["ms"] / 1e3) / 1e9
    print(json.dumps({"metric": "hoisted key-switched rotations/s (N=2^16, level 20)",
                      "value": B * R * args.steps / (ms / 1e3), "unit": "rotations/s", "higher_is_better": True,
                      "n_gpus": 1, "steps": args.steps, "ms_per_step": ms / args.steps,
                      "roofline_keyswitch": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                                             "frac": ach / hbm, "launches": t["count"], "avg_us": avg * 1e6,
                                             "algorithmic_bytes_per_launch": t["bytes"] / t["count"],
                                             "alu": {"achieved": prod, "peak": mac_peak, "unit": "G products/s",
                                                     "frac": prod / mac_peak}},
                      "kernel_time_ms": {"multsum": tr[0]["ms"], "ntt_fwd": tr[1]["ms"], "ntt_inv": tr[2]["ms"],
                                         "modup_bconv": tr[3]["ms"], "moddown_bconv": tr[4]["ms"]},
                      "conversions": {name: {"ms": t["ms"], "launches": t["count"],
                                             "algorithmic_gbs": t["bytes"] / (t["ms"] / 1e3) / 1e9 if t["ms"] else None}
                                      for name, t in (("modup_bconv", tr[3]), ("moddown_bconv", tr[4]))},
                      "config": {"workload": "%d ciphertexts x %d rotation steps, one Decompose per ciphertext" % (B, R),
                                 "multsum_variant": args.ms_variant},
                      "autotune": pk.he_autotune_log(ctx).splitlines()}),
          flush=True)
    for h in cts:
        pk.he_ct_free(h)
    pk.he_ctx_destroy(ctx)


# Table 3 (dh-BSGS rows): the paper's Z and T transform times of a 128x128
# matrix ciphertext, logN 15, 14 levels, Lattigo v4.1.0 on an AMD Ryzen 7
# 7735HS CPU (seconds; thread count not stated)
PAPER_TABLE3 = {("Z", 8, 0): 2.004, ("Z", 8, 64): 1.362, ("Z", 8, 32): 1.249,
                ("Z", 16, 0): 1.286, ("Z", 16, 64): 1.094, ("Z", 16, 32): 1.179,
                ("T", 8, 0): 1.049, ("T", 8, 64): 0.701, ("T", 8, 32): 0.652,
                ("T", 16, 0): 0.725, ("T", 16, 64): 0.572, ("T", 16, 32): 0.613}


def run_sweep(args):
    """Batched products/s of B identical-shape 128x128 products at N=2^16,
    level 20 (DMatrixMult), for B = 1, 2, 4, 8, 16, 32, against one
    he_hmatmul per product: how far batching amortises the key reads."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import workloads
    pk.build()
    n, n1, level = N_MAT, 16, 20
    ctx = pk.he_ctx_create(pk.he_params_default(2), 1000)
    tstream = torch.cuda.Stream()
    pk.he_ctx_set_stream(ctx, tstream.cuda_stream)
    pk.he_keygen(ctx, pk.he_rot_steps_for_matmul(n, n1, n1, 1 << 15), True)
    Bmax = 32
    mats = [workloads.matmul_pair(n, 10 * i) for i in range(Bmax)]
    cts = [(pk.he_encrypt_matrix(ctx, A, level, 2 * i), pk.he_encrypt_matrix(ctx, Bm, level, 2 * i + 1))
           for i, (A, Bm) in enumerate(mats)]

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(tstream)
        for _ in range(reps):
            fn()
        e1.record(tstream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def plain_one():
        pk.he_ct_free(pk.he_hmatmul(ctx, cts[0][0], cts[0][1], n, n1, n1))

    plain_one()
    plain_ms = timed(plain_one, max(1, args.steps))
    rows = []
    for B in (1, 2, 4, 8, 16, 32):
        jobs = [(a, b, n, n1, n1) for a, b in cts[:B]]

        def step():
            for o in pk.he_hmatmul_batch(jobs):
                pk.he_ct_free(o)

        for _ in range(2):
            step()
        ms = timed(step, max(1, args.steps))
        rows.append({"batch": B, "ms_per_step": ms, "matmul_per_s": B / (ms / 1e3),
                     "over_plain": (B / (ms / 1e3)) / (1e3 / plain_ms)})
    print(json.dumps({"metric": "HE 128x128 matmul/s batched vs plain (batch sweep)", "unit": "matmul/s",
                      "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
                      "plain": {"ms_per_product": plain_ms, "matmul_per_s": 1e3 / plain_ms},
                      "batched": rows,
                      "config": {"workload": "B identical-shape 128x128 products, N=2^16, q 60+20x40, p 2x60, "
                                             "level 20, n1_z=n1_t=16, DMatrixMult"}}), flush=True)
    pk.he_ctx_destroy(ctx)


def run_transforms(args):
    """The Z (sigma) and T (tau) transforms alone, as Table 3 measures them:
    one 128x128 matrix ciphertext at N = 2^15 (n^2 = slots, no replication),
    chain 60 + 14x40 with 2x60 special primes, n1 in {8, 16}, undecomposed
    (dh-BSGS) and with the Diagonal Convergence Decomposition at maximum
    diagonal 64 and 32 (depth 2 and 4), and with the simple key
    substitution of Sec. 4.2 (heads of 2 and 4 baby keys; Table 2 gives its
    key counts, Table 3 no times); the input level is chosen so that every
    run ends at level 10; device time per transform."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import workloads
    pk.build()
    ctx = pk.he_ctx_create(pk.make_params(15, [60] + [40] * 14, [60, 60]), 21)
    tstream = torch.cuda.Stream()
    pk.he_ctx_set_stream(ctx, tstream.cuda_stream)
    n, S = 128, 1 << 14
    steps = set()
    for n1 in (8, 16):
        for np_ in (0, 64, 32):
            steps |= set(pk.he_rot_steps_for_sched(n, n1, n1, S, np_, np_))
    pk.he_keygen(ctx, sorted(steps), False)     # covers the key-substitution heads too
    A, _ = workloads.matmul_pair(n, 5)
    info = pk.he_ctx_info(ctx)
    out = {}
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for name, kind in (("Z", 0), ("T", 1)):
        for n1 in (8, 16):
            for np_ in (0, 64, 32):
                depth = ((n - 1) if kind == 0 else (n - 2)) // np_ + 1 if np_ else 1
                ct = pk.he_encrypt_matrix(ctx, A, 10 + depth, 1)     # every run ends at level 10
                for _ in range(max(2, args.warmup)):
                    pk.he_ct_free(pk.he_linear_transform(ctx, ct, kind, n, n1, np_))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(tstream)
                for _ in range(args.steps):
                    pk.he_ct_free(pk.he_linear_transform(ctx, ct, kind, n, n1, np_))
                e1.record(tstream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                r = pk.he_linear_transform(ctx, ct, kind, n, n1, np_)
                d = pk.he_decrypt_matrix(ctx, r, n, n)
                ref = A[i, (i + j) % n] if kind == 0 else A[(i + j) % n, j]
                err = float(np.abs(d - ref).max())
                lv = pk.he_ct_info(r)[0]
                pk.he_ct_free(r)
                pk.he_ct_free(ct)
                # distinct rotation keys of the transform (Table 2): babies
                # 1..n1-1 plus the giants (and the +-n' / n'n steps of the
                # right factors under the decomposition)
                n2 = (np_ if np_ else n) // n1
                keys = (n1 + 2 * n2 - (1 if np_ else 2)) if kind == 0 else (n1 + n2 - (1 if np_ else 2))
                out["%s_n1_%d_maxdiag_%s" % (name, n1, np_ or "n-1")] = {
                    "ms": ms, "depth": depth, "end_level": lv, "max_abs_err": err,
                    "rotation_keys": keys, "paper_s": PAPER_TABLE3[(name, n1, np_)],
                    "speedup_vs_paper": PAPER_TABLE3[(name, n1, np_)] * 1e3 / ms}
    # Table 2's SmpKeySub rows (no Table 3 measurement in the paper): the
    # babies use only the keys of a head of n1' steps, depth 1
    for name, kind in (("Z", 0), ("T", 1)):
        for n1 in (8, 16):
            for head in (2, 4):
                ct = pk.he_encrypt_matrix(ctx, A, 11, 1)
                for _ in range(max(2, args.warmup)):
                    pk.he_ct_free(pk.he_linear_transform_ksub(ctx, ct, kind, n, n1, head))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(tstream)
                for _ in range(args.steps):
                    pk.he_ct_free(pk.he_linear_transform_ksub(ctx, ct, kind, n, n1, head))
                e1.record(tstream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                r = pk.he_linear_transform_ksub(ctx, ct, kind, n, n1, head)
                d = pk.he_decrypt_matrix(ctx, r, n, n)
                ref = A[i, (i + j) % n] if kind == 0 else A[(i + j) % n, j]
                err = float(np.abs(d - ref).max())
                lv = pk.he_ct_info(r)[0]
                pk.he_ct_free(r)
                pk.he_ct_free(ct)
                keys = len(pk.he_rot_steps_for_ksub(n, kind, n1, head, S))   # n^2 = slots: no replication step
                out["%s_n1_%d_ksub_head_%d" % (name, n1, head)] = {
                    "ms": ms, "depth": 1, "end_level": lv, "max_abs_err": err, "rotation_keys": keys}
    # one rotation key: dnum digits x 2 polys x (L+1+alpha) limbs x N words
    N, L, alpha, dnum = info["N"], info["L"], info["alpha"], info["dnum"]
    key_mb = dnum * 2 * (L + 1 + alpha) * N * 8 / 2 ** 20
    print(json.dumps({"metric": "Z / T linear transform time (Table 3 setting)", "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "results": out,
                      "rotation_key_mib": key_mb,
                      "paper_hardware": "Lattigo v4.1.0, AMD Ryzen 7 7735HS (CPU), logN 15, logQP 760, 14 levels",
                      "config": {"workload": "one 128x128 matrix ciphertext, N=2^15, q 60+14x40, p 2x60 "
                                             "(logQP 740), ends at level 10, n1 in {8, 16}, "
                                             "max diagonal n-1 / 64 / 32"}}), flush=True)
    pk.he_ctx_destroy(ctx)


def run_ntt(args):
    """The NTT alone (he_ntt) on R rows at N = 2^16 over the primes of the
    covariance chain at level 20 (R = 2024 is the forward transform of one
    batched Decompose of 8 products: 8 x 11 digits x 23 rows), device time of
    every launch from the library's CUDA-event trace, against the measured
    butterfly peak.  Also the small case for kernel profiles."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(2), 9)
    if args.ntt_variant is not None:
        pk.he_ctx_set_ntt_variant(ctx, args.ntt_variant)
    if args.ntt_chunk is not None:
        pk.he_ctx_set_ntt_chunk(ctx, args.ntt_chunk)
    tstream = torch.cuda.Stream()
    pk.he_ctx_set_stream(ctx, tstream.cuda_stream)
    q, p = pk.he_ctx_primes(ctx)
    primes = list(q) + list(p)
    R, N, level = args.ntt_rows, 1 << 16, 20
    rng = np.random.default_rng(12)
    host = np.stack([rng.integers(0, primes[r % len(primes)], N, dtype=np.uint64) for r in range(R)])
    dev = torch.from_numpy(host.view(np.int64)).cuda()
    del host
    for _ in range(max(3, args.warmup)):
        pk.he_ntt(ctx, dev.data_ptr(), R, level)
        pk.he_ntt(ctx, dev.data_ptr(), R, level, inverse=True)
    pk.he_trace_enable(ctx, True)
    for c in (1, 2):
        pk.he_trace_read(ctx, c, reset=True)
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        pk.he_ntt(ctx, dev.data_ptr(), R, level)
        pk.he_ntt(ctx, dev.data_ptr(), R, level, inverse=True)
    torch.cuda.nvtx.range_pop()
    tr = {c: pk.he_trace_read(ctx, c, reset=True) for c in (1, 2)}
    pk.he_trace_enable(ctx, False)
    peak = pk.he_bench_butterfly(4000) / 1e9
    hbm = peaks().get("hbm_gbs") or 6800.0
    out = {}
    for c, name in ((1, "forward"), (2, "inverse")):
        t = tr[c]
        # per transform of all R rows (a transform may run as several
        # launch pairs when the rows are chunked)
        avg = t["ms"] / args.steps / 1e3
        bfly = R * (N // 2) * 16 / avg / 1e9
        out[name] = {"avg_us": avg * 1e6, "gbfly_s": bfly, "frac_of_measured_peak": bfly / peak,
                     "launch_pairs_per_transform": t["count"] / args.steps,
                     "algorithmic_gbs": t["bytes"] / args.steps / avg / 1e9,
                     "hbm_frac_of_measured": t["bytes"] / args.steps / avg / 1e9 / hbm}
    print(json.dumps({"metric": "NTT butterflies/s (N=2^16, %d rows)" % R, "value": out["forward"]["gbfly_s"],
                      "unit": "Gbutterfly/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
                      "peak_gbfly_s": peak, "peak_source": "measured lazy-Shoup butterfly microbenchmark",
                      "forward": out["forward"], "inverse": out["inverse"],
                      "config": {"workload": "%d rows x 2^16 words, primes of q 60+20x40 and p 2x60 cycled"
                                             % R, "ntt_variant": args.ntt_variant, "ntt_chunk": args.ntt_chunk},
                      "traffic_note": "DRAM bytes per transform from ncu on the same command"}), flush=True)
    pk.he_ctx_destroy(ctx)


def run_mixed(args):
    """Config 4: 96 independent products, n in {16,32,64,128}, N in {2^15, 2^16},
    remaining level in [3, 20]; plain (one call each) vs one grouped batch."""
    import numpy as np
    import torch

    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300 import workloads
    pk.build()
    jobs = workloads.mixed_matmul_jobs(args.jobs, 4)
    ctxs = {15: pk.he_ctx_create(pk.he_params_default(4), 15), 16: pk.he_ctx_create(pk.he_params_default(2), 16)}
    for logN, ctx in ctxs.items():
        S = 1 << (logN - 1)
        steps = set()
        for n in sorted({j[0] for j in jobs if j[1] == logN}):
            steps |= set(pk.he_rot_steps_for_matmul(n, N1_FOR[n], N1_FOR[n], S))
        pk.he_keygen(ctx, sorted(steps), True)
    cts = []
    for i, (n, logN, level, A, B) in enumerate(jobs):
        ctx = ctxs[logN]
        cts.append((pk.he_encrypt_matrix(ctx, A, level, 2 * i), pk.he_encrypt_matrix(ctx, B, level, 2 * i + 1)))
    spec = [(a, b, n, N1_FOR[n], N1_FOR[n]) for (a, b), (n, _, _, _, _) in zip(cts, jobs)]
    outs = pk.he_hmatmul_batch(spec)            # warm-up: plaintext diagonals of every (n, level)
    for o in outs:
        pk.he_ct_free(o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [pk.he_hmatmul(ctxs[jobs[i][1]], cts[i][0], cts[i][1], jobs[i][0], N1_FOR[jobs[i][0]],
                           N1_FOR[jobs[i][0]]) for i in range(len(jobs))]
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = pk.he_hmatmul_batch(spec)
    t_batch = time.perf_counter() - t0
    # the whole mixed batch as one captured graph, every (N, level, n) group a
    # concurrent branch; creation (a recording run + capture) is not timed
    plan = pk.he_mm_plan_create(spec)
    for o in pk.he_mm_plan_run(plan):           # warm-up replay
        pk.he_ct_free(o)
    reps = max(1, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(reps):
        graph = pk.he_mm_plan_run(plan)
        if r + 1 < reps:
            for o in graph:
                pk.he_ct_free(o)
    t_graph = (time.perf_counter() - t0) / reps
    pinfo = pk.he_mm_plan_info(plan)
    bitexact = all(np.array_equal(pk.he_ct_export(ctxs[jobs[i][1]], plain[i]),
                                  pk.he_ct_export(ctxs[jobs[i][1]], batch[i])) and
                   np.array_equal(pk.he_ct_export(ctxs[jobs[i][1]], plain[i]),
                                  pk.he_ct_export(ctxs[jobs[i][1]], graph[i])) for i in range(len(jobs)))
    err = 0.0
    for i, (n, logN, level, A, B) in enumerate(jobs):
        err = max(err, float(np.abs(pk.he_decrypt_matrix(ctxs[logN], batch[i], n, n) - A @ B).max()))
    groups = len({(logN, level, n) for n, logN, level, _, _ in jobs})
    print(json.dumps({"metric": "mixed batch of encrypted matmuls/s (batched vs plain)",
                      "value": len(jobs) / t_graph, "unit": "matmul/s", "higher_is_better": True, "n_gpus": 1,
                      "plain": len(jobs) / t_plain, "speedup": t_plain / t_graph,
                      "graph": {"value": len(jobs) / t_graph, "ms_per_step": 1000 * t_graph,
                                "launches_per_step": pinfo["launches"], "plan_bytes": pinfo["bytes"],
                                "note": "one captured graph, every (N, level, n) group a concurrent branch"},
                      "grouped": {"value": len(jobs) / t_batch, "speedup_vs_plain": t_plain / t_batch,
                                  "note": "he_hmatmul_batch: groups one after another"},
                      "config": {"workload": "%d products, n in {16,32,64,128}, N in {2^15,2^16}, level in [3,20], "
                                             "chain 60+20x40, p 2x60" % len(jobs), "groups": groups},
                      "check": {"batch_and_graph_equal_plain_bitexact": bitexact, "max_abs_err_vs_fp64": err,
                                "tol": 1e-4}}),
          flush=True)
    for h in plain + batch + graph + [x for c in cts for x in c]:
        pk.he_ct_free(h)
    pk.he_mm_plan_destroy(plan)
    for ctx in ctxs.values():
        pk.he_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--preset", type=int, default=2, choices=[1, 2],
                    help="matmul: 2 = 128x128 at N=2^16 (the benchmark), 1 = 32x32 at N=2^14")
    ap.add_argument("--no-graph", action="store_true", help="matmul: skip the captured-graph replay")
    ap.add_argument("--no-once", action="store_true", help="matmul: skip the single-relinearisation measurement")
    ap.add_argument("--relin-once", action="store_true",
                    help="matmul: relinearise the summed tensors once per product (not the paper's DMatrixMult)")
    ap.add_argument("--n", type=int, default=N_MAT, choices=[16, 32, 64, 128],
                    help="matrix dimension (128 is the benchmark; smaller sizes are profiling cases)")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--oracle-full", action="store_true",
                    help="--impl reference: time the oracle on one whole 128x128 product (minutes)")
    ap.add_argument("--workload", default="matmul", choices=["matmul", "covariance", "pca", "mixed", "served", "ntt",
                                                           "keyswitch", "transforms", "sweep"])
    ap.add_argument("--ntt-rows", type=int, default=2024, help="ntt: rows transformed per launch")
    ap.add_argument("--rot-steps", type=int, default=8, help="keyswitch: rotation steps per ciphertext")
    ap.add_argument("--ntt-variant", type=int, default=None,
                    help="matmul / keyswitch / ntt: pin the NTT passes to one variant (default: the tuner)")
    ap.add_argument("--ntt-chunk", type=int, default=None,
                    help="ntt: rows per launch pair of the two-pass NTT (default: the tuner's)")
    ap.add_argument("--ms-variant", type=int, default=None,
                    help="matmul / keyswitch: pin every MultSum launch to one variant (default: the tuner)")
    ap.add_argument("--rate", type=float, default=4.0, help="served: arrivals per second")
    ap.add_argument("--duration", type=float, default=120.0, help="served: seconds of arrivals")
    ap.add_argument("--served-dcd", type=int, default=32,
                    help="served: maximum diagonal of the covariance products' decomposition (0: undecomposed)")
    ap.add_argument("--served-rows", type=int, default=60000,
                    help="served: rows of the dataset streamed as 128-row blocks (0: the older mix with products)")
    ap.add_argument("--budget-gb", type=float, default=200.0, help="served: device-memory budget of admitted jobs")
    ap.add_argument("--max-batch", type=int, default=8, help="served: products per batched pass")
    ap.add_argument("--no-pca", action="store_true", help="served: leave PCA jobs out of the mix")
    ap.add_argument("--no-compose", action="store_true", help="pca: skip the run with composite Newton steps")
    ap.add_argument("--jobs", type=int, default=96)
    ap.add_argument("--rows", type=int, default=256)
    ap.add_argument("--components", type=int, default=8)
    ap.add_argument("--pm-iters", type=int, default=14)
    args = ap.parse_args()
    if args.workload == "covariance":
        return run_covariance(args)
    if args.workload == "pca":
        return run_pca(args)
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "ntt":
        return run_ntt(args)
    if args.workload == "keyswitch":
        return run_keyswitch(args)
    if args.workload == "transforms":
        return run_transforms(args)
    if args.workload == "sweep":
        return run_sweep(args)
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(env_int("LOCAL_RANK", 0))
        tdist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
