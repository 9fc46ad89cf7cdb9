"""The single-key launch tuner (aes_autotune_blocks): the chosen kernel must be one of the
candidates, AES_IMPL_AUTO must then give the same bytes as every explicit kernel family (and
the oracle on sampled blocks), and the JSON cache must be written and reused."""
import json

import numpy as np
import pytest

from paper_1506_08503_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("key_bits", [128, 256])
def test_autotune_then_auto_matches(aes, orc, cuda, tmp_path, key_bits):
    import torch

    n = 1 << 22
    rng = np.random.default_rng(90 + key_bits)
    key = rng.integers(0, 256, key_bits // 8, dtype=np.uint8)
    ks = aes.aes_key_expand(key.tobytes(), key_bits)
    w = workloads.plain(91, n)
    x = torch.from_numpy(w.data).cuda()
    y = torch.empty_like(x)
    cache = tmp_path / "tune.json"
    for d in ("encrypt", "decrypt"):
        got = aes.aes_autotune_blocks(ks, x.data_ptr(), y.data_ptr(), n, d, cache)
        assert got["impl"] in ("ttable", "bitslice")
        again = aes.aes_autotune_blocks(ks, x.data_ptr(), y.data_ptr(), n, d, cache)  # from the cache
        assert again == got
        auto = aes.crypt(x, ks, d)
        for impl in ("ttable", "bitslice"):
            assert torch.equal(auto, aes.crypt(x, ks, d, impl=impl))
        idx = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 500)]))
        ti = torch.from_numpy(idx).cuda()
        torch.cuda.synchronize()
        sample = auto.view(-1, 16)[ti].cpu().numpy().reshape(-1)
        src = w.data.reshape(-1, 16)[idx].reshape(-1)
        want = (orc.encrypt_blocks if d == "encrypt" else orc.decrypt_blocks)(key, src, threads=8)
        assert (sample == want).all()
    entries = json.loads(cache.read_text())
    assert len(entries) == 2 and all("us" in v for v in entries.values())


def test_set_auto_choice_then_auto_matches(aes, cuda):
    import torch

    w = workloads.plain(92, 300_007)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = torch.from_numpy(w.data).cuda()
    ref = aes.crypt(x, ks, "encrypt", impl="ttable")
    for threads, u in ((768, 2), (256, 4), (512, 1)):
        aes.aes_set_auto_choice("encrypt", 10, "ttable", threads, u)
        assert torch.equal(aes.crypt(x, ks, "encrypt"), ref)
    aes.aes_set_auto_choice("encrypt", 10, "bitslice", 128, 32)
    assert torch.equal(aes.crypt(x, ks, "encrypt"), ref)
    # a pinned choice serves small calls too; cleared, small calls take the small-call kernel
    small = x[: 16 * 1000]
    assert torch.equal(aes.crypt(small, ks, "encrypt"), ref[: 16 * 1000])
    aes.aes_set_auto_choice("encrypt", 10, "auto", 0, 0)
    assert torch.equal(aes.crypt(small, ks, "encrypt"), ref[: 16 * 1000])
    assert torch.equal(aes.crypt(x, ks, "encrypt"), ref)
