"""ctypes binding of include/he.h (argument marshalling only).

Every function keeps the C name; all computation runs in libhe_gb300.so.
Loading fails loudly when the library is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhe_gb300.so")

HE_OK = 0
ERRORS = {
    -1: "HE_ERR_ARG", -2: "HE_ERR_PARAM", -3: "HE_ERR_LEVEL", -4: "HE_ERR_SCALE", -5: "HE_ERR_KEY_MISSING",
    -6: "HE_ERR_OOM", -7: "HE_ERR_ADMISSION", -8: "HE_ERR_TIMEOUT", -9: "HE_ERR_CUDA",
}
(HE_ERR_ARG, HE_ERR_PARAM, HE_ERR_LEVEL, HE_ERR_SCALE, HE_ERR_KEY_MISSING, HE_ERR_OOM, HE_ERR_ADMISSION,
 HE_ERR_TIMEOUT, HE_ERR_CUDA) = range(-1, -10, -1)


class HeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class he_params(ctypes.Structure):
    _fields_ = [("logN", ctypes.c_int), ("n_q", ctypes.c_int), ("q_bits", ctypes.c_int * 48),
                ("n_p", ctypes.c_int), ("p_bits", ctypes.c_int * 4), ("log_delta", ctypes.c_int),
                ("sigma", ctypes.c_double)]


class he_mm_sched(ctypes.Structure):
    _fields_ = [("n1_z", ctypes.c_int), ("n1_t", ctypes.c_int), ("relin_once", ctypes.c_int), ("dcd_z", ctypes.c_int),
                ("dcd_t", ctypes.c_int)]


class he_mm_job(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("n", ctypes.c_int), ("sched", he_mm_sched)]


class he_refresh_state(ctypes.Structure):
    _fields_ = [("next_obj", ctypes.c_uint32), ("count", ctypes.c_int)]


class he_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("max_batch", ctypes.c_int), ("reject_when_full", ctypes.c_int)]


class he_job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ctx", ctypes.c_void_p), ("in_", ctypes.POINTER(ctypes.c_void_p)),
                ("n_in", ctypes.c_int), ("n", ctypes.c_int), ("sched", he_mm_sched), ("n_row_blocks", ctypes.c_int),
                ("k", ctypes.c_int), ("s", ctypes.c_int), ("centered", ctypes.c_int), ("acc_id", ctypes.c_uint64),
                ("l_E", ctypes.c_int), ("l_P", ctypes.c_int), ("axis", ctypes.c_int),
                ("newton_counts", ctypes.POINTER(ctypes.c_int)), ("B2", ctypes.c_double),
                ("refresh_obj", ctypes.c_uint32)]


class he_serving_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in ("submitted", "admitted", "rejected", "completed", "failed",
                                                 "waited")] + \
               [(k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "jobs_per_s")] + \
               [(k, ctypes.c_longlong) for k in ("ticks", "products", "max_products_per_tick")] + \
               [(k, ctypes.c_double) for k in ("charged_bytes", "key_bytes")]


HE_JOB_MATMUL, HE_JOB_COVARIANCE, HE_JOB_XTX_BLOCK, HE_JOB_XTX_FINAL, HE_JOB_PCA = 1, 2, 3, 4, 5
HE_JOB_QUEUED, HE_JOB_RUNNING, HE_JOB_DONE, HE_JOB_FAILED, HE_JOB_WAITING = 0, 1, 2, 3, 4

P = ctypes.POINTER
vp = ctypes.c_void_p
ip = ctypes.c_int
u64p = P(ctypes.c_uint64)
dblp = P(ctypes.c_double)
i32p = P(ctypes.c_int32)
llp = P(ctypes.c_longlong)

# name -> argtypes (restype int unless listed in _RESTYPES)
SIGNATURES = {
    "he_last_error": [],
    "he_params_default": [ip, P(he_params)],
    "he_ctx_create": [P(he_params), ctypes.c_uint64, P(vp)],
    "he_ctx_destroy": [vp],
    "he_ctx_set_stream": [vp, vp],
    "he_ctx_primes": [vp, u64p, u64p],
    "he_ctx_set_autotune": [vp, ip],
    "he_ctx_set_multsum_variant": [vp, ip],
    "he_ctx_set_ntt_variant": [vp, ip],
    "he_ctx_set_ntt_chunk": [vp, ip],
    "he_ctx_set_newton_composition": [vp, ip],
    "he_ctx_set_packed_refresh": [vp, ip],
    "he_autotune_log": [vp, ctypes.c_char_p, ip, P(ip)],
    "he_ctx_info": [vp, P(ip), P(ip), P(ip), P(ip), P(ip)],
    "he_sk_export": [vp, P(ctypes.c_int64)],
    "he_keygen": [vp, i32p, ip, ip],
    "he_rot_steps_for_matmul": [ip, ip, ip, ip, i32p, P(ip)],
    "he_rot_steps_for_transpose": [ip, ip, ip, i32p, P(ip)],
    "he_rot_steps_for_sched": [ip, P(he_mm_sched), ip, i32p, P(ip)],
    "he_encrypt_slots": [vp, dblp, ip, ip, ctypes.c_uint64, P(vp)],
    "he_encrypt_matrix": [vp, dblp, ip, ip, ip, ctypes.c_uint64, P(vp)],
    "he_decrypt_slots": [vp, vp, dblp, ip],
    "he_decrypt_matrix": [vp, vp, dblp, ip, ip],
    "he_ct_info": [vp, P(ip), P(ctypes.c_double), P(ip)],
    "he_ct_export": [vp, u64p],
    "he_ct_import": [vp, u64p, ip, ctypes.c_double, ip, P(vp)],
    "he_ct_free": [vp],
    "he_rotate": [vp, vp, ip, P(vp)],
    "he_rotate_noalloc": [vp, vp, ip, ip, vp],
    "he_rotate_hoisted": [vp, P(vp), ip, i32p, ip, P(vp)],
    "he_add": [vp, vp, vp, P(vp)],
    "he_mult": [vp, vp, vp, P(vp)],
    "he_rescale": [vp, vp, P(vp)],
    "he_replicate": [vp, vp, ip, P(vp)],
    "he_hmatmul": [vp, vp, vp, ip, P(he_mm_sched), P(vp)],
    "he_hmatmul_batch": [P(he_mm_job), ip, P(vp)],
    "he_transpose": [vp, vp, ip, ip, ctypes.c_double, P(vp)],
    "he_linear_transform": [vp, vp, ip, ip, ip, ip, P(vp)],
    "he_refresh": [vp, vp, P(he_refresh_state), P(vp)],
    "he_aggregate": [vp, vp, ip, ip, P(vp)],
    "he_covariance": [vp, P(vp), ip, ip, ip, ip, ip, P(he_mm_sched), P(vp)],
    "he_covariance_partial": [vp, P(vp), ip, ip, ip, ip, ip, P(he_mm_sched), P(vp), P(vp)],
    "he_covariance_finish": [vp, P(vp), P(vp), ip, ip, ip, ip, P(he_mm_sched), ip, P(vp)],
    "he_lazy_normalization_schedule": [ip, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ip,
                                       P(ip)],
    "he_power_method": [vp, P(vp), ip, ip, P(vp), ip, ip, P(ip), ctypes.c_double, P(he_refresh_state), P(vp), P(vp), P(vp),
                        P(ip)],
    "he_eigen_shift": [vp, P(vp), ip, ip, vp, P(vp), ip, P(vp), P(he_refresh_state)],
    "he_pca": [vp, P(vp), ip, ip, ip, P(vp), ip, ip, P(ip), ctypes.c_double, P(he_refresh_state), P(vp), P(vp),
               P(ip)],
    "he_ntt": [vp, vp, ctypes.c_longlong, ip, ip],
    "he_linear_transform_ksub": [vp, vp, ip, ip, ip, ip, P(vp)],
    "he_rot_steps_for_ksub": [ip, ip, ip, ip, ip, i32p, P(ip)],
    "he_decompose": [vp, vp, ctypes.c_longlong, ip, vp],
    "he_moddown": [vp, vp, ctypes.c_longlong, ip, vp],
    "he_counters": [vp, llp, llp, llp, llp, ip],
    "he_trace_enable": [vp, ip],
    "he_bench_butterfly": [ip, P(ctypes.c_double)],
    "he_bench_mac": [ip, P(ctypes.c_double)],
    "he_trace_ops": [vp, ip, P(ctypes.c_double)],
    "he_trace_read": [vp, ip, llp, P(ctypes.c_double), P(ctypes.c_double), ip],
    "he_mm_plan_create": [P(he_mm_job), ip, P(vp)],
    "he_mm_plan_run": [vp, P(vp)],
    "he_mm_plan_info": [vp, llp, P(ctypes.c_double)],
    "he_mm_plan_destroy": [vp],
    "he_server_create": [P(he_server_cfg), P(vp), ip, P(vp)],
    "he_server_submit": [vp, P(he_job), P(ctypes.c_uint64)],
    "he_server_poll": [vp, ctypes.c_uint64, P(ip), P(ip), P(ctypes.c_double)],
    "he_server_wait": [vp, ctypes.c_uint64, ctypes.c_double, P(ip)],
    "he_server_result": [vp, ctypes.c_uint64, P(vp), ip, P(ip), P(ip), ip, P(ip)],
    "he_server_stats": [vp, ip, P(he_serving_stats)],
    "he_server_destroy": [vp],
}
_RESTYPES = {"he_last_error": ctypes.c_char_p}

_lib = None


def lib():
    """Load libhe_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhe_gb300.so not built: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, ctypes.c_int)
        _lib = L
    return _lib


def check(rc):
    if rc != HE_OK:
        raise HeError(rc, lib().he_last_error().decode())
    return rc


# ------------------------------------------------------------ wrappers
def he_params_default(cfg_id):
    p = he_params()
    check(lib().he_params_default(cfg_id, ctypes.byref(p)))
    return p


def make_params(logN, qbits, pbits, log_delta=40, sigma=3.2):
    p = he_params()
    p.logN = logN
    p.n_q = len(qbits)
    for i, b in enumerate(qbits):
        p.q_bits[i] = b
    p.n_p = len(pbits)
    for i, b in enumerate(pbits):
        p.p_bits[i] = b
    p.log_delta = log_delta
    p.sigma = sigma
    return p


def he_ctx_create(params, seed):
    h = vp()
    check(lib().he_ctx_create(ctypes.byref(params), seed, ctypes.byref(h)))
    return h


def he_ctx_destroy(ctx):
    check(lib().he_ctx_destroy(ctx))


def he_ctx_set_stream(ctx, stream_ptr):
    check(lib().he_ctx_set_stream(ctx, stream_ptr))


def he_ctx_set_autotune(ctx, on=True):
    check(lib().he_ctx_set_autotune(ctx, 1 if on else 0))


def he_ctx_set_multsum_variant(ctx, variant=-1):
    """Pins every MultSum launch to one variant (-1: tuner / defaults)."""
    check(lib().he_ctx_set_multsum_variant(ctx, int(variant)))


def he_ctx_set_ntt_variant(ctx, variant=-1):
    """Pins the NTT passes to one variant (-1: tuner)."""
    check(lib().he_ctx_set_ntt_variant(ctx, int(variant)))


def he_ctx_set_ntt_chunk(ctx, rows=0):
    """Rows per launch pair of the two-pass NTTs (0: all rows at once)."""
    check(lib().he_ctx_set_ntt_chunk(ctx, int(rows)))


def he_ctx_set_newton_composition(ctx, on=True):
    check(lib().he_ctx_set_newton_composition(ctx, 1 if on else 0))


def he_ctx_set_packed_refresh(ctx, on=True):
    check(lib().he_ctx_set_packed_refresh(ctx, 1 if on else 0))


def he_autotune_log(ctx):
    n = ctypes.c_int()
    check(lib().he_autotune_log(ctx, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    check(lib().he_autotune_log(ctx, buf, n.value + 1, None))
    return buf.value.decode()


def he_ctx_info(ctx):
    v = [ctypes.c_int() for _ in range(5)]
    check(lib().he_ctx_info(ctx, *[ctypes.byref(x) for x in v]))
    return dict(zip(["N", "slots", "L", "alpha", "dnum"], [x.value for x in v]))


def he_ctx_primes(ctx):
    info = he_ctx_info(ctx)
    q = np.zeros(info["L"] + 1, dtype=np.uint64)
    p = np.zeros(info["alpha"], dtype=np.uint64)
    check(lib().he_ctx_primes(ctx, q.ctypes.data_as(u64p), p.ctypes.data_as(u64p)))
    return [int(x) for x in q], [int(x) for x in p]


def he_sk_export(ctx):
    N = he_ctx_info(ctx)["N"]
    out = np.zeros(N, dtype=np.int64)
    check(lib().he_sk_export(ctx, out.ctypes.data_as(P(ctypes.c_int64))))
    return out


def he_keygen(ctx, steps, want_relin=True):
    a = np.ascontiguousarray(np.asarray(list(steps), dtype=np.int32))
    check(lib().he_keygen(ctx, a.ctypes.data_as(i32p), len(a), 1 if want_relin else 0))


def he_rot_steps_for_matmul(n, n1z, n1t, slots):
    out = np.zeros(4 * n + 64, dtype=np.int32)
    cnt = ctypes.c_int()
    check(lib().he_rot_steps_for_matmul(n, n1z, n1t, slots, out.ctypes.data_as(i32p), ctypes.byref(cnt)))
    return [int(x) for x in out[: cnt.value]]


def he_rot_steps_for_sched(n, n1z, n1t, slots, dcd_z=0, dcd_t=0):
    out = (ctypes.c_int32 * (8 * n + 64))()
    cnt = ctypes.c_int()
    s = he_mm_sched(n1z, n1t, 0, dcd_z, dcd_t)
    check(lib().he_rot_steps_for_sched(n, ctypes.byref(s), slots, out, ctypes.byref(cnt)))
    return list(out[:cnt.value])


def he_rot_steps_for_transpose(n, n1, slots):
    out = np.zeros(4 * n + 64, dtype=np.int32)
    cnt = ctypes.c_int()
    check(lib().he_rot_steps_for_transpose(n, n1, slots, out.ctypes.data_as(i32p), ctypes.byref(cnt)))
    return [int(x) for x in out[: cnt.value]]


def he_rot_steps_for_ksub(n, kind, n1, n1_sub, slots):
    """Slot rotation steps of sigma (kind 0) or tau (kind 1) with the simple
    key substitution of head length n1_sub (see include/he.h)."""
    cnt = ctypes.c_int(0)
    check(lib().he_rot_steps_for_ksub(n, kind, n1, n1_sub, slots, None, ctypes.byref(cnt)))
    out = np.zeros(max(1, cnt.value), dtype=np.int32)
    check(lib().he_rot_steps_for_ksub(n, kind, n1, n1_sub, slots, out.ctypes.data_as(i32p), ctypes.byref(cnt)))
    return [int(x) for x in out[: cnt.value]]


def he_linear_transform_ksub(ctx, ct, kind, n, n1, n1_sub):
    """sigma (kind 0) or tau (kind 1) with the simple key substitution."""
    h = vp()
    check(lib().he_linear_transform_ksub(ctx, ct, kind, n, n1, n1_sub, ctypes.byref(h)))
    return h


def he_encrypt_slots(ctx, z, level, enc_counter):
    z = np.ascontiguousarray(z, dtype=np.float64)
    h = vp()
    check(lib().he_encrypt_slots(ctx, z.ctypes.data_as(dblp), z.size, level, enc_counter, ctypes.byref(h)))
    return h


def he_encrypt_matrix(ctx, A, level, enc_counter):
    A = np.ascontiguousarray(A, dtype=np.float64)
    h = vp()
    check(lib().he_encrypt_matrix(ctx, A.ctypes.data_as(dblp), A.shape[0], A.shape[1], level, enc_counter,
                                  ctypes.byref(h)))
    return h


def he_decrypt_slots(ctx, ct, nslots):
    out = np.zeros(nslots, dtype=np.float64)
    check(lib().he_decrypt_slots(ctx, ct, out.ctypes.data_as(dblp), nslots))
    return out


def he_decrypt_matrix(ctx, ct, rows, cols):
    out = np.zeros((rows, cols), dtype=np.float64)
    check(lib().he_decrypt_matrix(ctx, ct, out.ctypes.data_as(dblp), rows, cols))
    return out


def he_ct_info(ct):
    lv, sc, per = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    check(lib().he_ct_info(ct, ctypes.byref(lv), ctypes.byref(sc), ctypes.byref(per)))
    return lv.value, sc.value, per.value


def he_ct_export(ctx, ct):
    lv, _, _ = he_ct_info(ct)
    N = he_ctx_info(ctx)["N"]
    out = np.zeros((2, lv + 1, N), dtype=np.uint64)
    check(lib().he_ct_export(ct, out.ctypes.data_as(u64p)))
    return out


def he_ct_import(ctx, residues, level, scale, period):
    r = np.ascontiguousarray(residues, dtype=np.uint64)
    h = vp()
    check(lib().he_ct_import(ctx, r.ctypes.data_as(u64p), level, scale, period, ctypes.byref(h)))
    return h


def he_ct_free(ct):
    check(lib().he_ct_free(ct))


def _unary(name, *args):
    h = vp()
    check(getattr(lib(), name)(*args, ctypes.byref(h)))
    return h


def he_rotate(ctx, ct, step):
    return _unary("he_rotate", ctx, ct, step)


def he_rotate_noalloc(ctx, in_dev_ptr, level, step, out_dev_ptr):
    """Rotation on caller-owned device buffers (raw device pointers as ints)."""
    check(lib().he_rotate_noalloc(ctx, vp(in_dev_ptr), level, step, vp(out_dev_ptr)))


def he_rotate_hoisted(ctx, cts, steps):
    """Returns outs[i][s] = Rot(cts[i], steps[s]) with one Decompose per ciphertext."""
    st = (ctypes.c_int32 * len(steps))(*steps)
    outs = (vp * (len(cts) * len(steps)))()
    check(lib().he_rotate_hoisted(ctx, _handles(cts), len(cts), st, len(steps), outs))
    return [[vp(outs[i * len(steps) + s]) for s in range(len(steps))] for i in range(len(cts))]


def he_add(ctx, a, b):
    return _unary("he_add", ctx, a, b)


def he_mult(ctx, a, b):
    return _unary("he_mult", ctx, a, b)


def he_rescale(ctx, a):
    return _unary("he_rescale", ctx, a)


def he_replicate(ctx, ct, n):
    return _unary("he_replicate", ctx, ct, n)


def he_hmatmul(ctx, A, B, n, n1z, n1t, relin_once=False, dcd_z=0, dcd_t=0):
    s = he_mm_sched(n1z, n1t, 1 if relin_once else 0, dcd_z, dcd_t)
    return _unary("he_hmatmul", ctx, A, B, n, ctypes.byref(s))


def he_hmatmul_batch(jobs):
    """jobs: list of (A, B, n, n1z, n1t[, relin_once])."""
    outs = (vp * len(jobs))()
    check(lib().he_hmatmul_batch(_mm_jobs(jobs), len(jobs), outs))
    return [vp(o) for o in outs]


def he_transpose(ctx, ct, n, n1, prescale=1.0):
    return _unary("he_transpose", ctx, ct, n, n1, prescale)


HE_LT_SIGMA, HE_LT_TAU, HE_LT_TRANSPOSE = 0, 1, 2


def he_linear_transform(ctx, ct, kind, n, n1, n_prime=0):
    return _unary("he_linear_transform", ctx, ct, kind, n, n1, n_prime)


def _handles(hs):
    arr = (vp * len(hs))()
    for i, h in enumerate(hs):
        arr[i] = h.value if isinstance(h, vp) else h
    return arr


def he_refresh(ctx, ct, rs):
    h = vp()
    check(lib().he_refresh(ctx, ct, ctypes.byref(rs), ctypes.byref(h)))
    return h


def he_aggregate(ctx, ct, axis, n):
    return _unary("he_aggregate", ctx, ct, axis, n)


def he_covariance_partial(ctx, blocks, n_row_blocks, k, n, s, centered, n1z, n1t, relin_once=False, dcd_z=0,
                          dcd_t=0):
    """One device's part of HCovMtrx over its row blocks ([l][j] order, l-major):
    returns (upper, colsum), upper the k(k+1)/2 sums X_a^T X_b / s (a <= b,
    row-major), colsum the k column sums ([] if centered)."""
    up = (vp * (k * (k + 1) // 2))()
    cs = (vp * k)()
    sc = he_mm_sched(n1z, n1t, 1 if relin_once else 0, dcd_z, dcd_t)
    check(lib().he_covariance_partial(ctx, _handles(blocks), n_row_blocks, k, n, s, 1 if centered else 0,
                                      ctypes.byref(sc), up, cs))
    return [vp(o) for o in up], ([] if centered else [vp(o) for o in cs])


def he_covariance_finish(ctx, upper, colsum, k, n, s, centered, n1z, n1t, block_level, relin_once=False, dcd_z=0,
                         dcd_t=0):
    """The k*k covariance blocks from summed parts (he_covariance_partial's outputs)."""
    out = (vp * (k * k))()
    sc = he_mm_sched(n1z, n1t, 1 if relin_once else 0, dcd_z, dcd_t)
    cs = _handles(colsum) if colsum else None
    check(lib().he_covariance_finish(ctx, _handles(upper), cs, k, n, s, 1 if centered else 0, ctypes.byref(sc),
                                     block_level, out))
    return [vp(o) for o in out]


def he_covariance(ctx, blocks, n_row_blocks, k, n, s, centered, n1z, n1t, relin_once=False, dcd_z=0, dcd_t=0):
    """blocks: list of handles in [l][j] order (l-major); returns k*k handles (a*k + b)."""
    out = (vp * (k * k))()
    sc = he_mm_sched(n1z, n1t, 1 if relin_once else 0, dcd_z, dcd_t)
    check(lib().he_covariance(ctx, _handles(blocks), n_row_blocks, k, n, s, 1 if centered else 0,
                              ctypes.byref(sc), out))
    return [vp(o) for o in out]


def he_lazy_normalization_schedule(t, S=0.5, e=1e-5, Bp=1e-3, B2=2.0 ** 16, max_iters=64):
    out = (ctypes.c_int * t)()
    check(lib().he_lazy_normalization_schedule(t, S, e, Bp, B2, max_iters, out))
    return list(out)


def he_power_method(ctx, cov, k, n, v0, axis, l_P, counts, B2, rs):
    lam = vp()
    V = (vp * k)()
    VT = (vp * k)()
    ax = ctypes.c_int()
    cs = (ctypes.c_int * len(counts))(*counts)
    check(lib().he_power_method(ctx, _handles(cov), k, n, _handles(v0), axis, l_P, cs, B2, ctypes.byref(rs),
                                ctypes.byref(lam), V, VT, ctypes.byref(ax)))
    return lam, [vp(x) for x in V], [vp(x) for x in VT], ax.value


def he_pca(ctx, cov, k, n, l_E, v0, axis, l_P, counts, B2, rs):
    """Returns (lambdas[l_E], V[l_E][k], axes[l_E])."""
    lams = (vp * l_E)()
    V = (vp * (l_E * k))()
    axes = (ctypes.c_int * l_E)()
    cs = (ctypes.c_int * len(counts))(*counts)
    check(lib().he_pca(ctx, _handles(cov), k, n, l_E, _handles(v0), axis, l_P, cs, B2, ctypes.byref(rs), lams, V,
                       axes))
    return ([vp(x) for x in lams], [[vp(V[m * k + j]) for j in range(k)] for m in range(l_E)], list(axes))


def he_eigen_shift(ctx, cov, k, n, lam, V, axis, VT, rs):
    """Shifts in place: returns the new list of k*k handles (the old ones are freed)."""
    arr = _handles(cov)
    check(lib().he_eigen_shift(ctx, arr, k, n, lam, _handles(V), axis, _handles(VT), ctypes.byref(rs)))
    return [vp(x) for x in arr]


TRACE_MULTSUM, TRACE_NTT_FWD, TRACE_NTT_INV = 0, 1, 2


def he_ntt(ctx, rows_dev_ptr, n_rows, level, inverse=False):
    """In-place NTT (or inverse) of n_rows device rows (see include/he.h)."""
    check(lib().he_ntt(ctx, rows_dev_ptr, n_rows, level, 1 if inverse else 0))


def he_decompose(ctx, poly_dev_ptr, n_items, level, digits_dev_ptr):
    """Decompose of n_items device polynomials into their extended digits (see include/he.h)."""
    check(lib().he_decompose(ctx, poly_dev_ptr, n_items, level, digits_dev_ptr))


def he_moddown(ctx, in_dev_ptr, n_items, level, out_dev_ptr):
    """Rounding ModDown of n_items device elements of Q_level P (see include/he.h)."""
    check(lib().he_moddown(ctx, in_dev_ptr, n_items, level, out_dev_ptr))


def he_trace_enable(ctx, on=True):
    check(lib().he_trace_enable(ctx, 1 if on else 0))


def he_bench_butterfly(iters=2000):
    v = ctypes.c_double()
    check(lib().he_bench_butterfly(iters, ctypes.byref(v)))
    return v.value


def he_trace_read(ctx, cls, reset=False):
    """Launches, device time (ms), algorithmic bytes and (MultSum) products of
    a traced kernel class since its last reset."""
    n, ms, by, ops = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib().he_trace_ops(ctx, cls, ctypes.byref(ops)))
    check(lib().he_trace_read(ctx, cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), 1 if reset else 0))
    return {"count": n.value, "ms": ms.value, "bytes": by.value, "ops": ops.value}


def he_bench_mac(iters=2000):
    v = ctypes.c_double()
    check(lib().he_bench_mac(iters, ctypes.byref(v)))
    return v.value


def he_counters(ctx, reset=False):
    v = [ctypes.c_longlong() for _ in range(4)]
    check(lib().he_counters(ctx, *[ctypes.byref(x) for x in v], 1 if reset else 0))
    return dict(zip(["MS", "Dp", "MD", "launches"], [x.value for x in v]))


# ------------------------------------------------------------- serving
def he_server_create(ctxs, hbm_budget_bytes, max_batch=8, reject_when_full=False):
    cfg = he_server_cfg(float(hbm_budget_bytes), max_batch, 1 if reject_when_full else 0)
    h = vp()
    check(lib().he_server_create(ctypes.byref(cfg), _handles(ctxs), len(ctxs), ctypes.byref(h)))
    return h


def he_server_submit(srv, kind, inputs=(), ctx=None, n=0, n1z=1, n1t=1, n_row_blocks=0, k=0, s=0, centered=False,
                     acc_id=0, l_E=0, l_P=0, axis=0, counts=None, B2=0.0, refresh_obj=0, relin_once=False,
                     dcd_z=0, dcd_t=0):
    """Queues one job (see include/he.h, he_job); returns its id.  Raises
    HeError (HE_ERR_ADMISSION when over the budget)."""
    arr = _handles(list(inputs)) if len(inputs) else None
    cs = (ctypes.c_int * len(counts))(*counts) if counts else None
    j = he_job(kind, ctx.value if isinstance(ctx, vp) else ctx,
               ctypes.cast(arr, P(vp)) if arr is not None else None, len(inputs), n,
               he_mm_sched(n1z, n1t, 1 if relin_once else 0, dcd_z, dcd_t),
               n_row_blocks, k, s, 1 if centered else 0, acc_id, l_E, l_P, axis,
               ctypes.cast(cs, P(ctypes.c_int)) if cs is not None else None, B2, refresh_obj)
    jid = ctypes.c_uint64()
    check(lib().he_server_submit(srv, ctypes.byref(j), ctypes.byref(jid)))
    return jid.value


def he_server_poll(srv, job_id):
    """Returns (status, error code, latency ms)."""
    st, err, lat = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    check(lib().he_server_poll(srv, job_id, ctypes.byref(st), ctypes.byref(err), ctypes.byref(lat)))
    return st.value, err.value, lat.value


def he_server_wait(srv, job_id, timeout_s=600.0):
    st = ctypes.c_int()
    check(lib().he_server_wait(srv, job_id, timeout_s, ctypes.byref(st)))
    return st.value


def he_server_result(srv, job_id, max_outs=256, max_aux=64):
    """Returns (outputs, aux); raises HeError with the job's code if it failed."""
    outs = (vp * max_outs)()
    aux = (ctypes.c_int * max_aux)()
    no, na = ctypes.c_int(), ctypes.c_int()
    check(lib().he_server_result(srv, job_id, outs, max_outs, ctypes.byref(no), aux, max_aux, ctypes.byref(na)))
    return [vp(outs[i]) for i in range(no.value)], list(aux[:na.value])


def he_server_stats(srv, kind=0):
    st = he_serving_stats()
    check(lib().he_server_stats(srv, kind, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in he_serving_stats._fields_}


def he_server_destroy(srv):
    check(lib().he_server_destroy(srv))


# ---------------------------------------------------------- graph plans
def _mm_jobs(jobs):
    """(A, B, n, n1z, n1t[, relin_once[, dcd_z, dcd_t]]) tuples -> he_mm_job array."""
    arr = (he_mm_job * len(jobs))()
    for i, j in enumerate(jobs):
        a, b, n, n1z, n1t = j[:5]
        once = 1 if len(j) > 5 and j[5] else 0
        dz, dt = (j[6], j[7]) if len(j) > 7 else (0, 0)
        arr[i] = he_mm_job(a.value if isinstance(a, vp) else a, b.value if isinstance(b, vp) else b, n,
                           he_mm_sched(n1z, n1t, once, dz, dt))
    return arr


def he_mm_plan_create(jobs):
    """jobs: list of (A, B, n, n1z, n1t); returns a plan handle."""
    h = vp()
    check(lib().he_mm_plan_create(_mm_jobs(jobs), len(jobs), ctypes.byref(h)))
    h.n_jobs = len(jobs)
    return h


def he_mm_plan_run(plan):
    outs = (vp * plan.n_jobs)()
    check(lib().he_mm_plan_run(plan, outs))
    return [vp(o) for o in outs]


def he_mm_plan_info(plan):
    n, b = ctypes.c_longlong(), ctypes.c_double()
    check(lib().he_mm_plan_info(plan, ctypes.byref(n), ctypes.byref(b)))
    return {"launches": n.value, "bytes": b.value}


def he_mm_plan_destroy(plan):
    check(lib().he_mm_plan_destroy(plan))

