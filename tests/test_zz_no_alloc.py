"""The rotation for callers that cannot allocate device memory.

he_rotate_noalloc works on device buffers the caller owns and keeps every
temporary in a fixed array the library reserves at load time.  Its output
must match he_rotate's, call after call, although all calls share that array.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc_vs_rotate(pk, ctx, cases, seed):
    """Runs he_rotate_noalloc and he_rotate on the same ciphertexts, one
    (level, step) case after the other, and compares the residues."""
    import torch

    N = pk.he_ctx_info(ctx)["N"]
    rng = np.random.default_rng(seed)
    for call, (level, step) in enumerate(cases):
        z = rng.uniform(-1, 1, N // 2)
        ct = pk.he_encrypt_slots(ctx, z, level, 500 + call)
        want_ct = pk.he_rotate(ctx, ct, step)
        want = pk.he_ct_export(ctx, want_ct)
        res = pk.he_ct_export(ctx, ct)
        d_in = torch.from_numpy(res.view(np.int64).copy()).cuda()
        d_out = torch.zeros_like(d_in)
        # the call runs on the context's stream: torch's writes must be done
        torch.cuda.synchronize()
        pk.he_rotate_noalloc(ctx, d_in.data_ptr(), level, step, d_out.data_ptr())
        got = d_out.cpu().numpy().view(np.uint64).reshape(want.shape)
        # the same integer arithmetic as he_rotate: the residues agree exactly
        assert np.array_equal(got, want), "call %d (level %d, step %d)" % (call, level, step)
        # and the rotated slots decrypt to rho(z; step)
        back = pk.he_ct_import(ctx, got, level, pk.he_ct_info(ct)[1], N // 2)
        assert np.abs(pk.he_decrypt_slots(ctx, back, N // 2) - np.roll(z, -step)).max() < 1e-5
        for h in (ct, want_ct, back):
            pk.he_ct_free(h)


def test_rotate_noalloc_matches_rotate_on_consecutive_calls():
    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(1), 31)
    try:
        pk.he_keygen(ctx, [3, 100], want_relin=False)
        _noalloc_vs_rotate(pk, ctx, [(3, 3), (1, 100), (3, 100)], 4)
    finally:
        pk.he_ctx_destroy(ctx)


def test_rotate_noalloc_two_special_primes_and_size_limit():
    """Two special primes (digits of two q's): level 3 has two full digits,
    level 4 ends with a digit of one prime; both fit the reserved array at
    N = 2^16 and equal he_rotate on consecutive calls.  Level 5 needs more
    temporaries than the array holds and is rejected with a clear error."""
    import torch

    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(2), 5)
    try:
        pk.he_keygen(ctx, [1, 16], want_relin=False)
        _noalloc_vs_rotate(pk, ctx, [(3, 1), (4, 16), (4, 1), (3, 16)], 8)
        words = 2 * 6 * (1 << 16)
        t = torch.zeros(words, dtype=torch.int64, device="cuda")
        u = torch.zeros(words, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        with pytest.raises(pk.HeError) as e:
            pk.he_rotate_noalloc(ctx, t.data_ptr(), 5, 1, u.data_ptr())
        assert "scratch" in str(e.value)
    finally:
        pk.he_ctx_destroy(ctx)
