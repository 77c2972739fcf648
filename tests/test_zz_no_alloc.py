"""The rotation for callers that cannot allocate device memory.

he_rotate_noalloc works on device buffers the caller owns and keeps every
temporary in a fixed array the library reserves at load time.  Its output
must match he_rotate's, call after call, although all calls share that array.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rotate_noalloc_matches_rotate_on_consecutive_calls():
    import torch

    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(1), 31)
    try:
        steps = [3, 100]
        pk.he_keygen(ctx, steps, want_relin=False)
        N = pk.he_ctx_info(ctx)["N"]
        rng = np.random.default_rng(4)
        for call, (level, step) in enumerate([(3, 3), (1, 100), (3, 100)]):
            z = rng.uniform(-1, 1, N // 2)
            ct = pk.he_encrypt_slots(ctx, z, level, 500 + call)
            want_ct = pk.he_rotate(ctx, ct, step)
            want = pk.he_ct_export(ctx, want_ct)
            res = pk.he_ct_export(ctx, ct)
            d_in = torch.from_numpy(res.view(np.int64).copy()).cuda()
            d_out = torch.zeros_like(d_in)
            pk.he_rotate_noalloc(ctx, d_in.data_ptr(), level, step, d_out.data_ptr())
            got = d_out.cpu().numpy().view(np.uint64).reshape(want.shape)
            # the same integer arithmetic as he_rotate: the residues agree exactly
            assert np.array_equal(got, want), "call %d" % call
            # and the rotated slots decrypt to rho(z; step)
            back = pk.he_ct_import(ctx, got, level, pk.he_ct_info(ct)[1], N // 2)
            assert np.abs(pk.he_decrypt_slots(ctx, back, N // 2) - np.roll(z, -step)).max() < 1e-5
            for h in (ct, want_ct, back):
                pk.he_ct_free(h)
        # sizes beyond the reserved scratch are rejected with a clear error
        with pytest.raises(pk.HeError) as e:
            big = pk.he_ctx_create(pk.he_params_default(2), 5)
            try:
                pk.he_keygen(big, [1], want_relin=False)
                words = 2 * 21 * (1 << 16)
                t = torch.zeros(words, dtype=torch.int64, device="cuda")
                pk.he_rotate_noalloc(big, t.data_ptr(), 20, 1, t.data_ptr() + 0)
            finally:
                pk.he_ctx_destroy(big)
        assert "scratch" in str(e.value)
    finally:
        pk.he_ctx_destroy(ctx)
