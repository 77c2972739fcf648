"""Plaintext pins of the matrix-multiplication transforms (no encryption):
the closed-form diagonals of eq. 5 / eq. 6 against the JKLS index maps, the
product identity eq. 4, the BSGS identity eq. 3', and the key / operation
counts of Table 1 and Table 3."""
import os

import numpy as np
import pytest

from oracle.hmm import diag_G, diag_T, diag_Z, mask_C, matmul_rot_steps, rot_slots


# JKLS index maps written from the matrix definitions (Sec. 3.4):
#   sigma(A)_{i,j} = A_{i,i+j}, tau(A)_{i,j} = A_{i+j,j},
#   phi^k(A)_{i,j} = A_{i,j+k}, psi^k(A)_{i,j} = A_{i+k,j}, G(A) = A^T.
def sigma(A):
    n = A.shape[0]
    return np.array([[A[i, (i + j) % n] for j in range(n)] for i in range(n)])


def tau(A):
    n = A.shape[0]
    return np.array([[A[(i + j) % n, j] for j in range(n)] for i in range(n)])


def phi(A, k):
    n = A.shape[0]
    return np.array([[A[i, (j + k) % n] for j in range(n)] for i in range(n)])


def psi(A, k):
    n = A.shape[0]
    return np.array([[A[(i + k) % n, j] for j in range(n)] for i in range(n)])


def apply_diagonals(diags, m):
    """eq. 2: U m = sum_t u_t . rho(m; t)."""
    out = np.zeros_like(m)
    for t, u in diags:
        out += u * rot_slots(m, t % m.size)
    return out


@pytest.mark.parametrize("n", [2, 3, 4, 8, 16])
def test_eq5_eq6_match_index_maps(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    a = A.ravel()
    Zd = [(k, diag_Z(n, k)) for k in range(-n + 1, n)]
    assert np.allclose(apply_diagonals(Zd, a), sigma(A).ravel())
    Td = [(k * n, diag_T(n, k * n)) for k in range(n)]
    assert np.allclose(apply_diagonals(Td, a), tau(A).ravel())
    Gd = [((n - 1) * k, diag_G(n, (n - 1) * k, n - 1)) for k in range(-n + 1, n)]
    assert np.allclose(apply_diagonals(Gd, a), A.T.ravel())
    for k in range(1, n):
        m1, m2 = mask_C(n, k)
        assert np.allclose(m1 * rot_slots(a, k) + m2 * rot_slots(a, (k - n) % (n * n)), phi(A, k).ravel())
        assert np.allclose(rot_slots(a, n * k), psi(A, k).ravel())
    # the number of non-zero diagonals (Sec. 4.1): 2n-1 for Z, n for T
    assert sum(1 for _, u in Zd if u.any()) == 2 * n - 1
    assert sum(1 for _, u in Td if u.any()) == n


@pytest.mark.parametrize("n", [2, 4, 8, 5])
def test_eq4_product_identity(n):
    rng = np.random.default_rng(10 + n)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    c = sum(phi(sigma(A), k).ravel() * psi(tau(B), k).ravel() for k in range(n))
    assert np.allclose(c, (A @ B).ravel())


def bsgs(diag, a, n, n1, giants, m):
    """eq. 3' (second line): sum_i rho( sum_j rho(u_{a(n1 i+j)}; -a n1 i) . rho(m; a j) ; a n1 i)."""
    n2 = n * n
    out = np.zeros_like(m)
    for i in giants:
        inner = np.zeros_like(m)
        for j in range(n1):
            u = diag(a * (n1 * i + j))
            if u is None:
                continue
            inner += rot_slots(u, (-a * n1 * i) % n2) * rot_slots(m, (a * j) % n2)
        out += rot_slots(inner, (a * n1 * i) % n2)
    return out


@pytest.mark.parametrize("n,n1", [(4, 2), (8, 2), (8, 4), (16, 4), (16, 8), (8, 8)])
def test_bsgs_identity(n, n1):
    rng = np.random.default_rng(n * 31 + n1)
    A = rng.standard_normal((n, n))
    a = A.ravel()
    n2 = n // n1
    assert np.allclose(bsgs(lambda t: diag_Z(n, t), 1, n, n1, range(-n2, n2), a), sigma(A).ravel())
    assert np.allclose(bsgs(lambda t: diag_T(n, t), n, n, n1, range(0, n2), a), tau(A).ravel())
    assert np.allclose(bsgs(lambda t: diag_G(n, t, n - 1), n - 1, n, n1, range(-n2, n2), a), A.T.ravel())


# ------------------------------------------------------- Table 1 / Table 3

def table1_keys(n, n1z, n1t):
    """MinRotKeys of the 'Optimized' rows of Table 1: Z n1+2n2-2, T n1+n2-2;
    C^k adds the step -n (its other keys are Z's), R^k adds none."""
    n2z, n2t = n // n1z, n // n1t
    return (n1z + 2 * n2z - 2), (n1t + n2t - 2)


@pytest.mark.parametrize("n,n1z,n1t", [(8, 2, 2), (16, 4, 4), (32, 8, 8), (128, 16, 16), (128, 8, 16)])
def test_key_set_matches_table1(n, n1z, n1t):
    S = n * n  # no replication steps
    steps = matmul_rot_steps(n, n1z, n1t, S)
    kz, kt = table1_keys(n, n1z, n1t)
    # Z's keys include the C^k extra step -n (= giant -n2z) and the chain step n1z (= giant 1);
    # T's keys include the R^k chain step n*n1t; Z and T keys are disjoint apart from
    # multiples of n that both use.
    zsteps = {j for j in range(1, n1z)} | {(n1z * i) % S for i in range(-(n // n1z), n // n1z) if i}
    tsteps = {(n * j) % S for j in range(1, n1t)} | {(n * n1t * i) % S for i in range(1, n // n1t)}
    assert len(zsteps) == kz and len(tsteps) == kt
    assert set(steps) == zsteps | tsteps


def test_table3_rotation_key_memory():
    # Table 3 (Sec. 7.1): Rtk(MB) of Z and T under dh-BSGS and DCDmp for a
    # 128x128 product at logN=15, 15 q's and 3 special primes.  Every row is
    # (MinRotKeys of Table 2 + 1 extra key) x one key of
    # 2 * dnum * (L+1+alpha) * N * 8 bytes = 2*5*18*2^15*8 B = 45 MiB.
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_rtk.txt")
    key_mib = 2 * 5 * 18 * (1 << 15) * 8 / (1 << 20)
    n = 128
    rows = 0
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        scheme, lt, n1, maxdiag, rtk = line.split()
        n1, maxdiag, rtk = int(n1), int(maxdiag), int(rtk)
        if scheme == "dh-BSGS":
            n2 = n // n1
            keys = n1 + 2 * n2 - 2 if lt == "Z" else n1 + n2 - 2
        else:  # DCDmp rows, Table 2: n1 + 2 n2' - 1 (Z), n1 + n2' - 1 (T), n2' = n'/n1
            n2p = maxdiag // n1
            keys = n1 + 2 * n2p - 1 if lt == "Z" else n1 + n2p - 1
        assert round((keys + 1) * key_mib) == rtk, line
        rows += 1
    assert rows == 12


# ---------------------------------------------------------------- DCD
@pytest.mark.parametrize("n,n_prime", [(8, 2), (8, 4), (16, 4), (16, 8), (32, 8),
                                       (4, 1), (8, 1), (8, 7), (16, 3), (16, 5), (16, 15)])
def test_dcd_factors_multiply_back_to_Z_and_T(n, n_prime):
    """Sec. 4.2: the factor chains of DCDforZ / DCDforT multiply (Boolean
    product) back to exactly the permutation matrices of eq. 5 / eq. 6; the
    right factors have only the diagonals 0 and +-n' (Z) or n' n (T); the left
    factor keeps diagonals inside [0, n'), (-n', 0] (Z) or {t n, t <= n'} (T);
    Z's chains have floor((n-1)/n') + 1 factors, T's floor((n-2)/n') + 1."""
    from oracle import dcd
    size = n * n
    z1, z2 = dcd.dcd_Z(n, n_prime)
    t = dcd.dcd_T(n, n_prime)
    assert len(z1) == len(z2) == (n - 1) // n_prime + 1 and len(t) == (n - 2) // n_prime + 1
    p1, p2 = dcd.chain_product(z1), dcd.chain_product(z2)
    assert not (p1 & p2) and (p1 | p2) == dcd.perm_entries(n, "Z")
    assert dcd.chain_product(t) == dcd.perm_entries(n, "T")
    # the same matrices from the closed forms of eq. 5 and eq. 6
    for k in range(-n + 1, n):
        u = diag_Z(n, k)
        got = dcd.diagonal(dcd.perm_entries(n, "Z"), size, k)
        assert np.array_equal(u, got)
    # right factors: diagonals 0 and +-n' (Z) or n' n (T) only (a late round
    # may have moved every entry, leaving no 0 diagonal)
    for f in z1[:-1]:
        assert n_prime in dcd.diagonal_set(f, size, True) and set(dcd.diagonal_set(f, size, True)) <= {0, n_prime}
    for f in z2[:-1]:
        assert -n_prime in dcd.diagonal_set(f, size, True) and set(dcd.diagonal_set(f, size, True)) <= {-n_prime, 0}
    for f in t[:-1]:
        assert n_prime * n in dcd.diagonal_set(f, size, False)
        assert set(dcd.diagonal_set(f, size, False)) <= {0, n_prime * n}
    assert all(0 <= k < n_prime for k in dcd.diagonal_set(z1[-1], size, True))
    assert all(-n_prime < k <= 0 for k in dcd.diagonal_set(z2[-1], size, True))
    assert all(k % n == 0 and k // n <= n_prime for k in dcd.diagonal_set(t[-1], size, False))


@pytest.mark.parametrize("n,n1,n_prime", [(16, 4, 8), (32, 4, 16), (128, 8, 64), (128, 8, 32), (128, 16, 64),
                                          (128, 16, 32)])
def test_dcd_key_sets_match_table2(n, n1, n_prime):
    """Table 2 DCDmp: MinRotKeys n1 + 2 n2' - 1 (Z) and n1 + n2' - 1 (T),
    n2' = n'/n1, counted on the actual step sets of the schedule."""
    from oracle.hmm import dcd_rot_steps
    z, t = dcd_rot_steps(n, n1, n1, n_prime, n_prime)
    n2p = n_prime // n1
    assert len(z) == n1 + 2 * n2p - 1
    assert len(t) == n1 + n2p - 1


def test_dcd_table3_key_memory_rows():
    """Table 3 DCDmp rows: (keys of the step sets + 1) x 45 MiB."""
    from oracle.hmm import dcd_rot_steps
    key_mib = 2 * 5 * 18 * (1 << 15) * 8 / (1 << 20)
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_rtk.txt")
    seen = 0
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line or not line.startswith("DCDmp"):
            continue
        _, lt, n1, maxdiag, rtk = line.split()
        z, t = dcd_rot_steps(128, int(n1), int(n1), int(maxdiag), int(maxdiag))
        keys = len(z) if lt == "Z" else len(t)
        assert round((keys + 1) * key_mib) == int(rtk), line
        seen += 1
    assert seen == 8


@pytest.mark.parametrize("n,n1", [(16, 4), (16, 8), (32, 8), (128, 8), (128, 16)])
def test_key_substitution_key_sets_match_table2(n, n1):
    """Table 2 SmpKeySub: MinRotKeys n1' + 2 n2 - 2 (Z) and n1' + n2 - 2 (T)
    for every head length 2 <= n1' <= n1, counted on the step sets the
    transforms use; n1' = n1 is the plain dh-BSGS row (n1 + 2 n2 - 2,
    n1 + n2 - 2)."""
    from oracle.hmm import ksub_rot_steps
    n2 = n // n1
    for n1p in range(2, n1 + 1):
        assert len(ksub_rot_steps(n, 0, n1, n1p)) == n1p + 2 * n2 - 2
        assert len(ksub_rot_steps(n, 1, n1, n1p)) == n1p + n2 - 2
