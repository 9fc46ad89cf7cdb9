"""Measurements behind the roofline and two design notes, run as GPU tests (print with -s).

* pipe rates: the integer issue rates (lanes per SM-clock) that the on-chip roofline in
  bench.py is built from, measured by the standalone program tests/probes/pipe_rates.cu
  (compiled here with nvcc; it is not part of the library);
* co-run: the T-table and bitsliced kernels on disjoint parts of one buffer at once, the
  premise of the combined roofline (bitsliced warps filling the ALU slots the T-table
  kernel leaves idle);
* host link: pinned host<->device copy rates, the bound of the end-to-end figures.

Each test prints one JSON line and checks only what must hold whatever the numbers are
(the program ran, the split output equals the unsplit one).
"""
import json
import shutil
import subprocess
import tempfile
import time
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

HERE = Path(__file__).resolve().parent


def test_pipe_rates(cuda):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = Path(d) / "pipe_rates"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", str(exe),
                        str(HERE / "probes" / "pipe_rates.cu")], check=True, capture_output=True, text=True)
        out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout
    res = json.loads(out)
    print(json.dumps({"probe": "pipe rates", "result": res}))
    for name, v in res.items():
        if isinstance(v, dict):
            assert 1.0 < v["lanes_per_sm_clock"] < 512.0, name


def test_corun_ttable_and_bitsliced(aes_lib_ready):
    """1 GiB AES-128 encryption split between the T-table kernel (first 1 - f) and the
    bitsliced kernel (last f) on two streams that start after the same event."""
    import torch

    aes = aes_lib_ready
    n = 1 << 26
    x = torch.randint(0, 256, (n * 16,), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    ks = aes.aes_key_expand(bytes(range(16)))
    main_s, sa, sb = torch.cuda.current_stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def launch(nt, nbs):
        sa.wait_stream(main_s)
        sb.wait_stream(main_s)
        aes.aes_crypt_blocks(ks, None, x.data_ptr(), y.data_ptr(), nt, "encrypt", "ttable", sa)
        if nbs:
            aes.aes_crypt_blocks(ks, None, x.data_ptr() + nt * 16, y.data_ptr() + nt * 16, nbs, "encrypt",
                                 "bitslice", sb)
        main_s.wait_stream(sa)
        main_s.wait_stream(sb)

    rows = []
    for share in (0.0, 0.05, 0.08, 0.10, 0.12, 0.15, 0.20):
        nbs = (int(n * share) // 1024) * 1024
        for _ in range(2):
            launch(n - nbs, nbs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main_s)
        for _ in range(20):
            launch(n - nbs, nbs)
        e1.record(main_s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        rows.append({"bitsliced_share": share, "ms_per_GiB": round(ms, 3), "gbps": round(n * 16 / ms / 1e6, 1)})
    z = torch.empty_like(x)
    aes.aes_crypt_blocks(ks, None, x.data_ptr(), z.data_ptr(), n, "encrypt", "ttable")
    launch(n - (n // 10 // 1024) * 1024, (n // 10 // 1024) * 1024)
    torch.cuda.synchronize()
    same = bool(torch.equal(z, y))
    print(json.dumps({"probe": "co-run", "rows": rows, "split_output_equals_ttable": same}))
    assert same
    del x, y, z
    torch.cuda.empty_cache()


def test_host_link(aes_lib_ready):
    """1 GiB pinned H2D, D2H and both at once over 1, 2, 4 and 8 streams (torch copies), and
    aes_crypt_host on pinned buffers."""
    import torch

    aes = aes_lib_ready
    n_bytes = 1 << 30
    hp = torch.randint(0, 256, (n_bytes,), dtype=torch.uint8).pin_memory()
    hq = torch.empty(n_bytes, dtype=torch.uint8).pin_memory()
    dg = torch.empty(n_bytes, dtype=torch.uint8, device="cuda")
    dh = torch.empty(n_bytes, dtype=torch.uint8, device="cuda")

    def rate(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return round(n_bytes * reps / (time.perf_counter() - t) / 1e9, 1)

    out = {}
    for k in (1, 2, 4, 8):
        streams = [torch.cuda.Stream() for _ in range(k)]
        chunk = n_bytes // k

        def h2d():
            for i, st in enumerate(streams):
                with torch.cuda.stream(st):
                    dg[i * chunk:(i + 1) * chunk].copy_(hp[i * chunk:(i + 1) * chunk], non_blocking=True)

        def d2h():
            for i, st in enumerate(streams):
                with torch.cuda.stream(st):
                    hq[i * chunk:(i + 1) * chunk].copy_(dh[i * chunk:(i + 1) * chunk], non_blocking=True)

        out[f"h2d_gbs_streams{k}"] = rate(h2d)
        out[f"d2h_gbs_streams{k}"] = rate(d2h)
        out[f"both_ways_gbs_each_streams{k}"] = rate(lambda: (h2d(), d2h()))
    ks = aes.aes_key_expand(bytes(16))
    out["aes_crypt_host_pinned_gbs"] = rate(
        lambda: aes.aes_crypt_host(ks, None, hp.data_ptr(), hq.data_ptr(), n_bytes // 16, "encrypt"), reps=3)
    print(json.dumps({"probe": "host link", "result": out}))
    assert all(v > 0 for v in out.values())
    del dg, dh
    torch.cuda.empty_cache()
