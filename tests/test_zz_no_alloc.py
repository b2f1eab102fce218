"""pc2_decrypt_noalloc: decryption for callers that may not allocate device
memory (fixed memory budgets, plugins kept away from the device allocator,
latency paths that cannot take an allocator's device-wide synchronisation).

Called through the C ABI and compared word for word with pc2_decrypt (the
results are integers, so the tolerance is exact equality), on two calls in a
row: the fixed scratch array keeps the first call's contents, and the second
call must not depend on them.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _fn():
    from paper_2601_14980_b300 import pc2

    f = pc2._lib.pc2_decrypt_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


# 3072 bits: two lanes per element, and 5000 elements exceed what the cut grid
# holds in one pass (58 CTAs x 64 elements), so the persistent loop runs.
@pytest.mark.parametrize("nbits,count", [(512, 1000), (1024, 1000), (2048, 20000), (3072, 5000)])
def test_decrypt_noalloc_matches_decrypt_twice(nbits, count):
    import torch

    from paper_2601_14980_b300 import pc2
    from paper_2601_14980_b300 import workloads as W

    torch.cuda.set_device(0)
    ctx = pc2.Context(0)
    key = pc2.Key.generate(nbits, 4242)
    fn = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        m = W.plaintexts_u64(count, seed=100 + call)
        dm = torch.from_numpy(m.view(np.int64)).cuda()
        ct = pc2.encrypt(ctx, key, dm, 777 + call, 3)
        ref = pc2.decrypt(ctx, key, ct, count)
        out = torch.full_like(ref, -1)
        assert fn(key.h, ct.data_ptr(), count, out.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        got = pc2.unpack(ctx, out, count, key.limbs)
        want = pc2.unpack(ctx, ref, count, key.limbs)
        assert torch.equal(got, want), "call %d differs from pc2_decrypt" % call
        # and it is the plaintext
        w = got.cpu().numpy().view(np.uint32).reshape(count, key.limbs)
        assert np.array_equal(w[:, 0].astype(np.uint64) | (w[:, 1].astype(np.uint64) << np.uint64(32)), m)
        assert not w[:, 2:].any()


def test_decrypt_noalloc_argument_errors():
    import torch

    from paper_2601_14980_b300 import pc2

    torch.cuda.set_device(0)
    key = pc2.Key.generate(512, 5)
    fn = _fn()
    buf = torch.zeros(pc2.tiled_words(1, 2 * key.limbs), dtype=torch.int32, device="cuda")
    assert fn(key.h, None, 1, buf.data_ptr(), None) == -1          # PC2_EINVAL
    assert fn(key.public().h, buf.data_ptr(), 1, buf.data_ptr(), None) == -3   # PC2_EKEY
    assert fn(key.h, buf.data_ptr(), 0, buf.data_ptr(), None) == 0  # nothing to do
