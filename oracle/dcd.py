"""Diagonal Convergence Decomposition of Z and T (Sec. 4.2) -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Matrices here are n^2 x n^2 Boolean matrices given as sets of (row, column)
entries.  The diagonal of entry (r, c) is k = c - r (Definition 3), taken in
(-n^2/2, n^2/2] for Z and in [0, n^2) for T.  Decomposing diagonal k onto
diagonal k_r of a right factor and k_l = k - k_r of a left factor
(Definition 4) puts, for every entry (r, c) on it, the entry (c - k_r, c) in
the right factor (same column) and (r, r + k_l) in the left one (same row),
so that left * right reproduces the entry through the middle index
a = r + k_l = c - k_r (Theorem 2).

Readings:
  * a diagonal with |k| >= n' (Z) goes to k_r = sign(k) n'; the others keep
    k_l = k, k_r = 0 (DCDforZ, Sec. 4.2).  The prose of that section uses a
    strict comparison and names diagonal n' of the left factor as the target,
    and a left part n' with a right part sign(k) n' would not add up to k, so
    the algorithm's own steps are taken;
  * T: diagonals t n with t <= n' stay (k_r = 0), the others move by n' n
    (DCDforT);
  * rounds, each applied to the previous left factor, so Z_t = L R_m ...
    R_1 with R_1 applied first to the vector: Z takes floor((n-1)/n') rounds
    (its left factor must keep |k| < n', the range of its BSGS), T takes
    floor((n-2)/n') (its left factor may keep t = n'); both give n/n'
    factors for n' | n (Table 2).  With ceil((n-1)/n') - 1 rounds for Z, an
    n' dividing n - 1 (n1 = 1 with an odd n') would leave diagonal n' in the
    left factor, outside its BSGS range.
"""
import numpy as np


def perm_entries(n, which):
    """Entries of Z (sigma, eq. 5) or T (tau, eq. 6) on row-major n x n
    slots: output slot l = i n + j reads input slot sigma(l) / tau(l)."""
    l = np.arange(n * n)
    i, j = l // n, l % n
    src = i * n + (i + j) % n if which == "Z" else ((i + j) % n) * n + j
    return {(int(r), int(c)) for r, c in zip(l, src)}


def diag_index(r, c, size, centred):
    k = (c - r) % size
    if centred and k > size // 2:
        k -= size
    return k


def split_step(entries, size, pick, centred):
    """One decomposition round: entries = left * right with pick(k) ->
    (k_left, k_right), k_left + k_right = k."""
    left, right = set(), set()
    for r, c in entries:
        kl, kr = pick(diag_index(r, c, size, centred))
        right.add(((c - kr) % size, c))
        left.add((r, (r + kl) % size))
    return left, right


def bool_product(left, right):
    """Entries of left * right over the Boolean semiring."""
    by_row = {}
    for a, c in right:
        by_row.setdefault(a, []).append(c)
    out = set()
    for r, a in left:
        for c in by_row.get(a, ()):
            out.add((r, c))
    return out


def rounds(n, n_prime, which="Z"):
    return (n - 1) // n_prime if which == "Z" else (n - 2) // n_prime


def chain_length(n, n_prime, which="Z"):
    """Factors (levels) of the decomposed Z or T."""
    return rounds(n, n_prime, which) + 1


def dcd_Z(n, n_prime):
    """DCDforZ: Z = Z_1 + Z_2 (diagonals >= 0 / < 0), each a chain of factors
    in application order [R_1, ..., R_{m-1}, L]."""
    size = n * n
    full = perm_entries(n, "Z")
    parts = ({e for e in full if diag_index(*e, size, True) >= 0},
             {e for e in full if diag_index(*e, size, True) < 0})

    def pick(k):
        if abs(k) >= n_prime:
            s = 1 if k > 0 else -1
            return k - s * n_prime, s * n_prime
        return k, 0

    chains = []
    for part in parts:
        cur, rights = part, []
        for _ in range(rounds(n, n_prime)):
            cur, r = split_step(cur, size, pick, True)
            rights.append(r)
        chains.append(rights + [cur])
    return chains


def dcd_T(n, n_prime):
    """DCDforT: T as one chain of factors in application order."""
    size = n * n

    def pick(k):
        t = k // n
        return (k, 0) if t <= n_prime else (k - n_prime * n, n_prime * n)

    cur, rights = perm_entries(n, "T"), []
    for _ in range(rounds(n, n_prime, "T")):
        cur, r = split_step(cur, size, pick, False)
        rights.append(r)
    return rights + [cur]


def chain_product(chain):
    """The matrix a chain applies: the last factor times ... times the first."""
    out = chain[0]
    for f in chain[1:]:
        out = bool_product(f, out)
    return out


def diagonal(entries, size, k):
    """Slot vector of diagonal k of a factor (eq. 2): u_k[r] = M[r, r + k]."""
    u = np.zeros(size)
    for r, c in entries:
        if (c - r) % size == k % size:
            u[r] = 1.0
    return u


def diagonal_set(entries, size, centred):
    return sorted({diag_index(r, c, size, centred) for r, c in entries})
