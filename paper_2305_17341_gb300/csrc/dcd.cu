// dcd.cu -- the Diagonal Convergence Decomposition of the Z and T transforms
// (Sec. 4.2, Definition 4, Theorem 2, DCDforZ, DCDforT), built on the host
// once per (transform, n, n') and kept on the device as per-row diagonal
// tables of its factors.
//
// A factor is an n^2 x n^2 Boolean matrix with at most one entry per row; it
// is stored as col[r] (-1 for an empty row).  Decomposing the diagonal
// k = c - r of an entry (r, c) onto the diagonal k_r of a right factor and
// k_l = k - k_r of a left factor places (c - k_r, c) in the right factor and
// (r, r + k_l) in the left one: left * right reproduces the entry through the
// middle index r + k_l = c - k_r.  Z splits into Z_1 (diagonals >= 0) and Z_2
// (< 0); a diagonal with |k| >= n' moves by sign(k) n', the others stay on
// the left factor.  T's diagonals t n with t > n' move by n' n.  After
// Z_t = L R_m ... R_1 after floor((n-1)/n') rounds for Z (its left factor
// must keep |k| < n', the range of its BSGS) and floor((n-2)/n') for T (its
// left factor may keep t = n'): n/n' factors for n' | n (Table 2).
#include <set>
#include <sstream>
#include <stdexcept>

#include "eval.h"

namespace he {

namespace {

typedef std::vector<int> Factor;   // col[r], -1 = empty row

long centred(long k, long size) {
    k %= size;
    if (k < 0) k += size;
    return k > size / 2 ? k - size : k;
}

// One round: cur = left * right for the given split of each entry's diagonal.
template <typename Pick>
void split(const Factor &cur, long size, bool centre, Pick pick, Factor &left, Factor &right) {
    left.assign(size, -1);
    right.assign(size, -1);
    for (long r = 0; r < size; r++) {
        if (cur[r] < 0) continue;
        const long c = cur[r];
        long k = (c - r) % size;
        if (k < 0) k += size;
        if (centre) k = centred(k, size);
        long kl, kr;
        pick(k, kl, kr);
        const long rr = ((c - kr) % size + size) % size, lc = ((r + kl) % size + size) % size;
        if (right[rr] >= 0 || left[r] >= 0) throw std::logic_error("decomposition collides");
        right[rr] = (int)c;
        left[r] = (int)lc;
    }
}

std::vector<Factor> chain(const Factor &start, long size, bool centre, int rounds,
                          void (*pick)(long, long, long &, long &), long arg) {
    std::vector<Factor> out;
    Factor cur = start, l, r;
    for (int i = 0; i < rounds; i++) {
        split(cur, size, centre, [&](long k, long &kl, long &kr) { pick(k, arg, kl, kr); }, l, r);
        out.push_back(r);
        cur = l;
    }
    out.push_back(cur);
    return out;
}

void pick_z(long k, long np, long &kl, long &kr) {
    if (k >= np || -k >= np) {
        const long s = k > 0 ? 1 : -1;
        kl = k - s * np, kr = s * np;
    } else {
        kl = k, kr = 0;
    }
}

// arg packs n' and n for T
void pick_t(long k, long arg, long &kl, long &kr) {
    const long np = arg >> 20, n = arg & ((1L << 20) - 1);
    if (k / n <= np) kl = k, kr = 0;
    else kl = k - np * n, kr = np * n;
}

__global__ void k_dcd_fill(double *out, int S, const int *diag, int n, long t, long rot, double value) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S) return;
    long n2 = (long)n * n;
    long l = ((long)(p % n2) + rot) % n2;
    long tt = ((t % n2) + n2) % n2;
    out[p] = diag[l] == tt ? value : 0.0;
}

}  // namespace

void launch_dcd_fill(Ctx *c, double *out, const int *diag, int n, long t, long rot, double value, cudaStream_t st) {
    c->n_launch++;
    k_dcd_fill<<<(c->S + 255) / 256, 256, 0, st>>>(out, c->S, diag, n, t, rot, value);
}

const DcdChain &dcd_chain(Ctx *c, int which, int n, int n_prime) {
    std::ostringstream os;
    os << "dcd:" << which << ':' << n << ':' << n_prime;
    const std::string key = os.str();
    auto it = c->dcd.find(key);
    if (it != c->dcd.end()) return it->second;
    if (n_prime < 1 || n_prime >= n) throw HeError(HE_ERR_ARG, "the decomposition needs 1 <= n' < n");
    const long size = (long)n * n;
    const int rounds = dcd_levels(n, n_prime, which == 2) - 1;
    // eq. 5 / eq. 6 on row-major slots: row l = i n + j
    Factor full(size);
    for (long l = 0; l < size; l++) {
        const long i = l / n, j = l % n;
        full[l] = which == 2 ? (int)(((i + j) % n) * n + j) : (int)(i * n + (i + j) % n);
    }
    std::vector<Factor> fs;
    if (which == 2) {
        fs = chain(full, size, false, rounds, pick_t, ((long)n_prime << 20) | n);
    } else {
        Factor part(size, -1);
        for (long r = 0; r < size; r++) {
            const long k = centred(full[r] - r, size);
            if ((which == 0) == (k >= 0)) part[r] = full[r];
        }
        fs = chain(part, size, true, rounds, pick_z, n_prime);
    }
    DcdChain ch;
    for (size_t f = 0; f < fs.size(); f++) {
        DcdFactor fac;
        std::vector<int> dg(size, -1);
        for (long r = 0; r < size; r++) {
            if (fs[f][r] < 0) continue;
            long k = ((fs[f][r] - r) % size + size) % size;
            dg[r] = (int)k;
            fac.diags.insert(k);
        }
        std::ostringstream fid;
        fid << key << ':' << f;
        fac.id = fid.str();
        if (cudaMalloc(&fac.dev, size * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            throw HeError(HE_ERR_OOM, "decomposition table allocation failed");
        }
        cudaMemcpy(fac.dev, dg.data(), size * sizeof(int), cudaMemcpyHostToDevice);
        if (f + 1 < fs.size()) {
            for (long k : fac.diags)
                if (k != 0) fac.step = k;
        }
        ch.factors.push_back(fac);
    }
    return c->dcd.emplace(key, std::move(ch)).first->second;
}

int dcd_levels(int n, int n_prime, bool is_t) {
    if (!n_prime) return 1;
    return (is_t ? (n - 2) / n_prime : (n - 1) / n_prime) + 1;
}

}  // namespace he
