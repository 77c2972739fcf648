"""ctypes bindings of oracle.c.  Test infrastructure only (see oracle/__init__.py)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)
u32p = ctypes.POINTER(ctypes.c_uint32)
dblp = ctypes.POINTER(ctypes.c_double)
intp = ctypes.POINTER(ctypes.c_int)


def build(force=False):
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_is_prime.argtypes = [ctypes.c_uint64]
            L.or_is_prime.restype = ctypes.c_int
            L.or_powmod.argtypes = [ctypes.c_uint64] * 3
            L.or_powmod.restype = ctypes.c_uint64
            L.or_invmod.argtypes = [ctypes.c_uint64] * 2
            L.or_invmod.restype = ctypes.c_uint64
            L.or_gen_primes.argtypes = [ctypes.c_int, ctypes.c_int, intp, ctypes.c_int, intp, u64p, u64p]
            L.or_gen_primes.restype = ctypes.c_int
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_sample_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, u64p]
            L.or_sample_ternary.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_int, i64p]
            L.or_sample_gauss.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_double, ctypes.c_int, i64p]
            L.or_gauss_table.argtypes = [ctypes.c_double, u64p]
            L.or_polymul_schoolbook.argtypes = [ctypes.c_uint64, ctypes.c_int, u64p, u64p, u64p]
            L.or_polymul.argtypes = [ctypes.c_uint64, ctypes.c_int, u64p, u64p, u64p]
            L.or_polymul_sum.argtypes = [ctypes.c_int, ctypes.c_int, u64p, ctypes.c_int, u64p, u64p, u64p]
            L.or_mulconst_limbs.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p, u64p, u64p]
            L.or_bconv.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p, ctypes.c_int, u64p, u64p]
            L.or_moddown_round.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p, ctypes.c_int, u64p, u64p, u64p]
            L.or_encode.argtypes = [ctypes.c_int, dblp, dblp, ctypes.c_double, i64p]
            L.or_decode.argtypes = [ctypes.c_int, dblp, ctypes.c_double, dblp, dblp]
            L.or_encode_direct.argtypes = [ctypes.c_int, dblp, dblp, ctypes.c_double, dblp]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a


def is_prime(n):
    return bool(lib().or_is_prime(int(n)))


def powmod(a, e, q):
    return int(lib().or_powmod(int(a), int(e), int(q)))


def invmod(a, q):
    return int(lib().or_invmod(int(a) % int(q), int(q)))


def gen_primes(logN, qbits, pbits):
    qb = (ctypes.c_int * len(qbits))(*qbits)
    pb = (ctypes.c_int * max(1, len(pbits)))(*pbits)
    oq = np.zeros(len(qbits), dtype=np.uint64)
    op = np.zeros(max(1, len(pbits)), dtype=np.uint64)
    rc = lib().or_gen_primes(logN, len(qbits), qb, len(pbits), pb, _p(oq, u64p), _p(op, u64p))
    if rc != 0:
        raise ValueError("prime search failed")
    return [int(x) for x in oq], [int(x) for x in op[:len(pbits)]]


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def sample_uniform(seed, obj, tag, limb, q, N):
    out = np.zeros(N, dtype=np.uint64)
    lib().or_sample_uniform(seed, obj, tag, limb, q, N, _p(out, u64p))
    return out


def sample_ternary(seed, obj, tag, N):
    out = np.zeros(N, dtype=np.int64)
    lib().or_sample_ternary(seed, obj, tag, N, _p(out, i64p))
    return out


def sample_gauss(seed, obj, tag, sigma, N):
    out = np.zeros(N, dtype=np.int64)
    lib().or_sample_gauss(seed, obj, tag, sigma, N, _p(out, i64p))
    return out


def gauss_table(sigma):
    out = np.zeros(20, dtype=np.uint64)
    lib().or_gauss_table(sigma, _p(out, u64p))
    return out


def polymul_schoolbook(q, a, b):
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    lib().or_polymul_schoolbook(q, a.size, _p(a, u64p), _p(b, u64p), _p(out, u64p))
    return out


def polymul(q, a, b):
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    lib().or_polymul(q, a.size, _p(a, u64p), _p(b, u64p), _p(out, u64p))
    return out


def polymul_sum(qs, a, b):
    """a, b: [nterms][nlimbs][N]; returns [nlimbs][N] = sum_t a[t]*b[t] per limb."""
    a, b = _u64(a), _u64(b)
    nterms, nl, N = a.shape
    assert b.shape == a.shape and len(qs) == nl
    qa = _u64(np.array(qs, dtype=np.uint64))
    out = np.zeros((nl, N), dtype=np.uint64)
    lib().or_polymul_sum(N, nl, _p(qa, u64p), nterms, _p(a, u64p), _p(b, u64p), _p(out, u64p))
    return out


def mulconst_limbs(qs, a, c):
    a = _u64(a)
    nl, N = a.shape
    qa = _u64(np.array(qs, dtype=np.uint64))
    ca = _u64(np.array([int(x) % int(q) for x, q in zip(c, qs)], dtype=np.uint64))
    out = np.zeros_like(a)
    lib().or_mulconst_limbs(N, nl, _p(qa, u64p), _p(a, u64p), _p(ca, u64p), _p(out, u64p))
    return out


def bconv(src_q, src, dst_q):
    src = _u64(src)
    ns, N = src.shape
    sq = _u64(np.array(src_q, dtype=np.uint64))
    dq = _u64(np.array(dst_q, dtype=np.uint64))
    out = np.zeros((len(dst_q), N), dtype=np.uint64)
    lib().or_bconv(N, ns, _p(sq, u64p), _p(src, u64p), len(dst_q), _p(dq, u64p), _p(out, u64p))
    return out


def moddown_round(qs, uQ, ps, uP):
    """round(X / P) over the q's for X given by residues uQ (q's) and uP (p's)."""
    uQ, uP = _u64(uQ), _u64(uP)
    nq, N = uQ.shape
    qa = _u64(np.array(qs, dtype=np.uint64))
    pa = _u64(np.array(ps, dtype=np.uint64))
    out = np.zeros_like(uQ)
    lib().or_moddown_round(N, nq, _p(qa, u64p), _p(uQ, u64p), len(ps), _p(pa, u64p), _p(uP, u64p),
                           _p(out, u64p))
    return out


def encode(z, N, scale):
    z = np.asarray(z)
    zr = np.ascontiguousarray(np.real(z), dtype=np.float64)
    zi = np.ascontiguousarray(np.imag(z), dtype=np.float64)
    assert zr.size == N // 2
    out = np.zeros(N, dtype=np.int64)
    lib().or_encode(N, _p(zr, dblp), _p(zi, dblp), float(scale), _p(out, i64p))
    return out


def encode_direct(z, N, scale):
    z = np.asarray(z)
    zr = np.ascontiguousarray(np.real(z), dtype=np.float64)
    zi = np.ascontiguousarray(np.imag(z), dtype=np.float64)
    out = np.zeros(N, dtype=np.float64)
    lib().or_encode_direct(N, _p(zr, dblp), _p(zi, dblp), float(scale), _p(out, dblp))
    return out


def decode(coef, scale):
    c = np.ascontiguousarray(coef, dtype=np.float64)
    N = c.size
    zr = np.zeros(N // 2)
    zi = np.zeros(N // 2)
    lib().or_decode(N, _p(c, dblp), float(scale), _p(zr, dblp), _p(zi, dblp))
    return zr + 1j * zi
