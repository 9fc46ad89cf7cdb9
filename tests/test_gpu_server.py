"""The continuous-batching server through the C ABI: correctness of every request against the
oracle, the same result alone and in a concurrent mix, backpressure, bounded waits, and
host-side fault injection (a launch that fails on the host, never on the GPU)."""
import os
import time

import numpy as np
import pytest

import paper_1506_08503_gb300 as aes

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


def make_pool(rng, n128=4, n256=4):
    keys128 = rng.integers(0, 256, (n128, 16), dtype=np.uint8)
    keys256 = rng.integers(0, 256, (n256, 32), dtype=np.uint8)
    pool = aes.KeyPool(n128 + n256)
    pool.load_keys(0, keys128, 128)
    pool.load_keys(n128, keys256, 256)
    return pool, [k for k in keys128] + [k for k in keys256]


def oracle_crypt(orc, key, data, d):
    return (orc.encrypt_blocks if d == 0 else orc.decrypt_blocks)(key, data, threads=THREADS)


def test_requests_match_oracle_host_and_device_buffers(aes_lib_ready, orc):
    import torch

    rng = np.random.default_rng(40)
    pool, keys = make_pool(rng)
    with pool, aes.Server(pool, hbm_budget=64 << 20, nstreams=4, max_batch=64) as srv:
        reqs = []
        for i in range(240):
            n = int(rng.integers(1, 2000))
            data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
            k, d = int(rng.integers(0, len(keys))), int(rng.integers(0, 2))
            mode = i % 4  # host->host, host->device, device->host, device->device
            src = torch.from_numpy(data).cuda() if mode >= 2 else data
            dst = torch.empty(16 * n, dtype=torch.uint8, device="cuda") if mode in (1, 3) else np.empty_like(data)
            torch.cuda.synchronize()
            sp = src.data_ptr() if mode >= 2 else src.ctypes.data
            dp = dst.data_ptr() if mode in (1, 3) else dst.ctypes.data
            t = srv.submit(k, d, sp, dp, 16 * n, mode >= 2, mode in (1, 3))
            reqs.append((t, data, src, dst, k, d, mode))
        for t, data, src, dst, k, d, mode in reqs:
            assert srv.poll(t, 10_000_000) == aes.AES_REQ_DONE
            got = dst.cpu().numpy() if mode in (1, 3) else dst
            assert (got == oracle_crypt(orc, keys[k], data, d)).all()
        st = srv.stats()
        assert st["completed"] == 240 and st["failed"] == 0 and st["queued"] == 0 and st["inflight"] == 0
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
        assert st["launches"] >= 1 and st["mean_batch"] >= 1


def test_host_buffers_staged_and_direct(aes_lib_ready, orc):
    """Host payloads 16-byte aligned (read and written by the kernel itself where the device
    reaches host memory directly) and 8 bytes off (copied through the staging arena), in every
    combination for source and destination, in one mix."""
    rng = np.random.default_rng(46)
    pool, keys = make_pool(rng)
    with pool, aes.Server(pool, hbm_budget=64 << 20, nstreams=4, max_batch=32) as srv:
        items = []
        for i in range(160):
            n = int(rng.integers(1, 3000))
            data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
            so, do = 8 * (i % 2), 8 * ((i // 2) % 2)
            src_buf = np.empty(16 * n + 16, dtype=np.uint8)
            dst_buf = np.empty(16 * n + 16, dtype=np.uint8)
            src_buf[so:so + 16 * n] = data
            k, d = int(rng.integers(0, len(keys))), int(rng.integers(0, 2))
            t = srv.submit(k, d, src_buf.ctypes.data + so, dst_buf.ctypes.data + do, 16 * n, False, False)
            items.append((t, data, src_buf, dst_buf, do, k, d))
        for t, data, src_buf, dst_buf, do, k, d in items:
            assert srv.poll(t, 10_000_000) == aes.AES_REQ_DONE
            assert (dst_buf[do:do + data.size] == oracle_crypt(orc, keys[k], data, d)).all()
        st = srv.stats()
        assert st["completed"] == 160 and st["failed"] == 0


def test_result_is_the_same_alone_and_in_the_mix(aes_lib_ready):
    import torch

    rng = np.random.default_rng(41)
    pool, keys = make_pool(rng)
    probe = rng.integers(0, 256, 16 * 5000, dtype=np.uint8)
    with pool, aes.Server(pool, hbm_budget=256 << 20, nstreams=4, max_batch=256) as srv:
        alone = np.empty_like(probe)
        t = srv.submit(5, 0, probe.ctypes.data, alone.ctypes.data, probe.size, False, False)
        assert srv.poll(t) == aes.AES_REQ_DONE
        # the same request inside a stream of 600 others of every size and direction, arriving
        # in two waves: the probe heads the second wave, queued while the first is on the GPU
        mixed = np.empty_like(probe)
        others = []
        for i in range(600):
            a = rng.integers(0, 256, 16 * int(rng.integers(1, 4000)), dtype=np.uint8)
            others.append((int(rng.integers(0, 8)), int(rng.integers(0, 2)), a, np.empty_like(a)))
        reqs = np.zeros(601, dtype=aes.request_dtype())
        rows = [(k, d, a.ctypes.data, b.ctypes.data, a.size) for k, d, a, b in others]
        rows.insert(300, (5, 0, probe.ctypes.data, mixed.ctypes.data, probe.size))
        cols = list(zip(*rows))
        for name, col in zip(("key_idx", "dir", "src", "dst", "length"), cols):
            reqs[name] = np.array(col, dtype=reqs.dtype[name])
        tickets = list(srv.submit_many(reqs[:300])) + list(srv.submit_many(reqs[300:]))
        for t in tickets:
            assert srv.poll(int(t)) == aes.AES_REQ_DONE
        assert (alone == mixed).all()
        # and the same as the plain single-key entry point
        ks = aes.aes_key_expand(keys[5].tobytes())
        x = torch.from_numpy(probe).cuda()
        assert (aes.encrypt(x, ks).cpu().numpy() == alone).all()
        assert srv.stats()["mean_batch"] > 1  # requests really were batched together


def test_backpressure_and_bounded_waits(aes_lib_ready):
    rng = np.random.default_rng(42)
    pool, keys = make_pool(rng)
    with pool, aes.Server(pool, hbm_budget=8 << 20, nstreams=1, max_batch=2, queue_capacity=3) as srv:
        bufs = [(rng.integers(0, 256, 16 * 20000, dtype=np.uint8), np.empty(16 * 20000, dtype=np.uint8))
                for _ in range(40)]
        outstanding, done, rejected, nsub = [], 0, 0, 0
        while nsub < 40:
            a, b = bufs[nsub]
            t = srv.try_submit(0, 0, a.ctypes.data, b.ctypes.data, a.size, False, False)
            if t is None:  # AES_EAGAIN: release the oldest ticket, then retry
                rejected += 1
                assert srv.poll(outstanding.pop(0)) == aes.AES_REQ_DONE
                done += 1
                continue
            outstanding.append(t)
            nsub += 1
        assert rejected > 0  # the holding limit was reached and submit said AES_EAGAIN
        for t in outstanding:
            assert srv.poll(t) == aes.AES_REQ_DONE
        assert done + len(outstanding) == 40
        # bounded wait on a request that cannot be finished in 0 us
        big = rng.integers(0, 256, 8 << 20, dtype=np.uint8)
        out = np.empty_like(big)
        t = srv.submit(1, 1, big.ctypes.data, out.ctypes.data, big.size, False, False)
        first = srv.poll(t, 0)
        assert first in (aes.AES_REQ_PENDING, aes.AES_REQ_DONE)
        if first == aes.AES_REQ_PENDING:
            assert srv.poll(t, -1) == aes.AES_REQ_DONE
        with pytest.raises(aes.AesError) as ei:
            srv.poll(t, 0)  # released after DONE was reported
        assert ei.value.status == aes.AES_ENOTFOUND
        with pytest.raises(aes.AesError) as ei:
            srv.poll(123456789, 0)
        assert ei.value.status == aes.AES_ENOTFOUND
        # a request larger than the whole staging budget is refused up front (a buffer 8 bytes
        # off 16-byte alignment is always staged, also where kernels reach host memory directly)
        huge = np.empty(16 << 20, dtype=np.uint8)
        with pytest.raises(aes.AesError) as ei:
            srv.submit(0, 0, huge.ctypes.data + 8, huge.ctypes.data + 8, huge.size - 16, False, False)
        assert ei.value.status == aes.AES_ENOMEM
        for bad in [(99, 0, 64), (0, 2, 64), (0, 0, 24), (0, 0, 0)]:
            with pytest.raises(aes.AesError) as ei:
                srv.submit(bad[0], bad[1], huge.ctypes.data, huge.ctypes.data, bad[2], False, False)
            assert ei.value.status == aes.AES_EINVAL


def test_injected_launch_failures_are_reported_and_contained(aes_lib_ready, orc):
    rng = np.random.default_rng(43)
    pool, keys = make_pool(rng)
    with pool, aes.Server(pool, hbm_budget=32 << 20, nstreams=1, max_batch=1, fail_every=3) as srv:
        items = []
        for i in range(30):
            a = rng.integers(0, 256, 16 * 100, dtype=np.uint8)
            b = np.zeros_like(a)
            items.append((srv.submit(i % 8, 0, a.ctypes.data, b.ctypes.data, a.size, False, False), a, b, i % 8))
        states = [srv.poll(t) for t, *_ in items]
        assert states.count(aes.AES_REQ_FAILED) == 10 and states.count(aes.AES_REQ_DONE) == 20
        for (t, a, b, k), s in zip(items, states):
            if s == aes.AES_REQ_DONE:
                assert (b == orc.encrypt_blocks(keys[k], a, threads=THREADS)).all()
        st = srv.stats()
        assert st["failed"] == 10 and st["completed"] == 20 and st["inflight"] == 0


def test_destroy_with_queued_work(aes_lib_ready):
    rng = np.random.default_rng(44)
    pool, keys = make_pool(rng)
    with pool:
        srv = aes.Server(pool, hbm_budget=16 << 20, nstreams=1, max_batch=1)
        keep = []
        for _ in range(50):
            a = rng.integers(0, 256, 1 << 20, dtype=np.uint8)
            b = np.empty_like(a)
            keep.append((a, b))
            srv.submit(0, 0, a.ctypes.data, b.ctypes.data, a.size, False, False)
        srv.close()  # fails what is still queued, drains the GPU, joins the thread


def test_submit_many_is_all_or_nothing(aes_lib_ready, orc):
    import torch

    rng = np.random.default_rng(45)
    pool, keys = make_pool(rng)
    with pool, aes.Server(pool, hbm_budget=64 << 20, nstreams=2, max_batch=512, queue_capacity=1000) as srv:
        n = 300
        lengths = rng.integers(1, 500, n) * 16
        offs = np.concatenate([[0], np.cumsum(lengths)[:-1]])
        data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
        src = torch.from_numpy(data).cuda()
        dst = torch.empty_like(src)
        torch.cuda.synchronize()
        reqs = np.zeros(n, dtype=aes.request_dtype())
        reqs["key_idx"] = rng.integers(0, 8, n)
        reqs["dir"] = rng.integers(0, 2, n)
        reqs["length"] = lengths
        reqs["src"], reqs["dst"] = src.data_ptr() + offs, dst.data_ptr() + offs
        reqs["src_on_device"] = reqs["dst_on_device"] = 1
        bad = reqs.copy()
        bad[150]["length"] = 24  # one bad request: nothing is queued
        with pytest.raises(aes.AesError) as ei:
            srv.submit_many(bad)
        assert ei.value.status == aes.AES_EINVAL and "request 150" in str(ei.value)
        assert srv.stats()["submitted"] == 0
        with pytest.raises(aes.AesError) as ei:
            srv.submit_many(np.concatenate([reqs] * 4))  # 1200 > queue capacity 1000
        assert ei.value.status == aes.AES_EAGAIN
        tickets = srv.submit_many(reqs)
        assert (np.diff(tickets.astype(np.int64)) == 1).all()
        assert all(srv.poll(int(t)) == aes.AES_REQ_DONE for t in tickets)
        got = dst.cpu().numpy()
        for i in range(n):
            o, L = int(offs[i]), int(lengths[i])
            f = orc.encrypt_blocks if reqs[i]["dir"] == 0 else orc.decrypt_blocks
            assert (got[o:o + L] == f(keys[int(reqs[i]["key_idx"])], data[o:o + L], threads=THREADS)).all(), i
        st = srv.stats()
        assert st["completed"] == n and st["mean_batch"] > 2


def test_trickled_requests_all_complete_without_a_lost_wakeup(aes_lib_ready, orc):
    """Requests submitted one at a time with irregular gaps (from none to a few hundred
    microseconds), so that the server's thread keeps switching between sleeping (nothing in
    flight) and polling its batches' done events: every request completes within a bounded
    wait, with the oracle's bytes."""
    import torch

    rng = np.random.default_rng(43)
    pool, keys = make_pool(rng)
    n = 1500
    lengths = 16 * rng.integers(1, 300, n)
    offs = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
    src = torch.from_numpy(data).cuda()
    dst = torch.empty_like(src)
    kidx = rng.integers(0, 8, n)
    dirs = rng.integers(0, 2, n)
    gaps = rng.choice([0.0, 0.0, 20e-6, 200e-6], n)
    with pool, aes.Server(pool, hbm_budget=64 << 20, nstreams=4, max_batch=64) as srv:
        tickets = []
        for i in range(n):
            if gaps[i]:
                end = time.perf_counter() + gaps[i]
                while time.perf_counter() < end:
                    pass
            o = int(offs[i])
            tickets.append(srv.submit(int(kidx[i]), int(dirs[i]), src.data_ptr() + o, dst.data_ptr() + o,
                                      int(lengths[i]), True, True))
        for t in tickets:
            assert srv.poll(t, timeout_us=5_000_000) == aes.AES_REQ_DONE
        st = srv.stats()
        assert st["completed"] == n and st["failed"] == 0
    got = dst.cpu().numpy()
    for i in rng.choice(n, 60, replace=False):
        o, L = int(offs[i]), int(lengths[i])
        assert (got[o:o + L] == oracle_crypt(orc, keys[int(kidx[i])], data[o:o + L], int(dirs[i]))).all(), i


def test_small_batches_take_the_one_launch_path(aes_lib_ready, orc):
    """Batches of at most 16 requests and 32768 blocks run as one kernel with their descriptors
    as launch parameters and the tables read from global memory: AES-128/192/256 keys, both
    directions, device and host payloads in one batch, against the oracle; a batch just over
    the limit takes the batched graph path and gives the same bytes."""
    import torch

    rng = np.random.default_rng(49)
    bits = [128, 192, 256, 128, 256, 192]
    keys = [rng.integers(0, 256, b // 8, dtype=np.uint8) for b in bits]
    pool = aes.KeyPool(len(keys))
    for i, k in enumerate(keys):
        pool.set(i, aes.aes_key_expand(k.tobytes(), 8 * len(k)))
    with pool, aes.Server(pool, hbm_budget=64 << 20, nstreams=2, max_batch=64) as srv:
        for count, max_blocks in ((10, 300), (16, 2048), (17, 100), (3, 12000)):
            lengths = rng.integers(1, max_blocks, count) * 16
            offs = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
            data = rng.integers(0, 256, int(lengths.sum()), dtype=np.uint8)
            src = torch.from_numpy(data).cuda()
            dst = torch.zeros_like(src)
            hdst = np.zeros_like(data)
            torch.cuda.synchronize()
            reqs = np.zeros(count, dtype=aes.request_dtype())
            reqs["key_idx"] = rng.integers(0, len(keys), count)
            reqs["dir"] = rng.integers(0, 2, count)
            reqs["length"] = lengths
            reqs["src"] = src.data_ptr() + offs
            on_host = np.arange(count) % 3 == 2  # every third output goes to host memory
            reqs["dst"] = np.where(on_host, hdst.ctypes.data + offs, dst.data_ptr() + offs)
            reqs["src_on_device"] = 1
            reqs["dst_on_device"] = np.where(on_host, 0, 1)
            tickets = srv.submit_many(reqs)
            assert all(srv.poll(int(t)) == aes.AES_REQ_DONE for t in tickets)
            got_dev = dst.cpu().numpy()
            for i in range(count):
                o, L = int(offs[i]), int(lengths[i])
                got = hdst[o:o + L] if on_host[i] else got_dev[o:o + L]
                want = oracle_crypt(orc, keys[int(reqs[i]["key_idx"])], data[o:o + L], int(reqs[i]["dir"]))
                assert (got == want).all(), (count, i)


def test_linger_keeps_worker_polling_and_results_exact(aes_lib_ready, orc):
    """A server whose worker keeps polling for 3 ms after its last request (linger_us): requests
    spaced 0.5 ms apart (inside the window) and 8 ms apart (after it, so the worker has gone to
    sleep and must be woken) all complete with the oracle's output, and the server shuts down
    cleanly while lingering."""
    import time

    import torch

    rng = np.random.default_rng(49)
    pool, keys = make_pool(rng)
    with pool, aes.Server(pool, hbm_budget=16 << 20, nstreams=2, max_batch=16, linger_us=3000) as srv:
        for gap in [0.0005] * 6 + [0.008] * 3 + [0.0005] * 3:
            n = int(rng.integers(1, 300))
            data = rng.integers(0, 256, 16 * n, dtype=np.uint8)
            k, d = int(rng.integers(0, len(keys))), int(rng.integers(0, 2))
            src = torch.from_numpy(data).cuda()
            dst = torch.empty_like(src)
            torch.cuda.synchronize()
            t = srv.submit(k, d, src.data_ptr(), dst.data_ptr(), 16 * n, True, True)
            assert srv.poll(t, 10_000_000) == aes.AES_REQ_DONE
            assert (dst.cpu().numpy() == oracle_crypt(orc, keys[k], data, d)).all()
            time.sleep(gap)
        st = srv.stats()
        assert st["completed"] == 12 and st["failed"] == 0
