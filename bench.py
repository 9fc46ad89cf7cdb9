#!/usr/bin/env python
"""Throughput benchmark: AES-128 encryption and decryption of many independent 16-byte
blocks on one GB300 (or N, one process each, under torchrun).

Workload (one "step"): expand one AES-128 key, encrypt a 1 GiB buffer of 2^26 uniform random
blocks (seed 1) and decrypt the ciphertext back, through the C ABI (aes_key_expand,
aes_encrypt_blocks, aes_decrypt_blocks).  Inputs are resident in HBM when the timed region
starts; the buffer (1 GiB) is larger than the 129 MB L2, so no flush is needed between steps.
`value` is bytes encrypted plus bytes decrypted per second over all ranks (GB/s, 1e9).

Also printed on the same JSON line:
  e2e           the same step on pinned HOST buffers through aes_crypt_host (copies in the
                timed region)
  roofline      the dominant kernel's achieved GB/s against the on-chip integer roofline
  cpu_baseline  the CPU oracle on the host cores, on a bounded sample of the same workload
  clocks        nvidia-smi SM clocks sampled during the timed region

`--impl reference` times the CPU oracle instead (the slow program the paper's method is
checked against), on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1506_08503_gb300 import workloads  # noqa: E402

METRIC = "AES-128 encrypt+decrypt throughput, many independent 16-byte blocks"
UNIT = "GB/s"
WORKLOAD = "aes128-enc+dec-1GiB-2^26-blocks-seed1"
NBLOCKS = 1 << 26
SEED = 1

# On-chip integer roofline ("Roofline"): per SM and clock the GB300 issues
# 64 lanes of integer ALU work (LOP3/PRMT/SHF/IADD, measured) and 32 lanes of shared-memory
# loads.  A table-lookup AES-128 block needs at least 160 lookups and 240 ALU operations; a
# gate-level (bitsliced) block at least 356.25 ALU lane-operations (22,800 two-input gates,
# two per LOP3, 32 blocks per lane).  Filling the LDS pipe with lookups and the ALU pipe's
# remainder with gates gives 0.2449 blocks per SM-clock.
ALU_LANES, LDS_LANES = 64.0, 32.0
TT_LDS, TT_ALU, BS_ALU = 160.0, 240.0, 22800.0 / 64.0
SM_COUNT_NOMINAL, SM_MAX_MHZ_NOMINAL = 152, 2070.0


def blocks_per_sm_clock() -> float:
    t = min(LDS_LANES / TT_LDS, ALU_LANES / TT_ALU)
    b = max(0.0, (ALU_LANES - TT_ALU * t) / BS_ALU)
    return t + b


def roofline_peak_gbs(sms: int, mhz: float) -> float:
    return blocks_per_sm_clock() * sms * mhz * 1e6 * 16 / 1e9


# ---------------------------------------------------------------------------------------------

def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--kernel", choices=["auto", "ttable", "bitslice"], default="auto")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle sample")
    p.add_argument("--nblocks", type=int, default=NBLOCKS, help="blocks per rank (default 2^26 = 1 GiB)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class Clocks:
    """nvidia-smi sampler, started before and stopped after a timed region."""

    FIELDS = ("index,timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None

    def mark(self, which: str):
        setattr(self, which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        self.file.flush()
        rows = []
        for line in Path(self.file.name).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                main_ts, _, frac = parts[1].partition(".")
                ts = time.mktime(time.strptime(main_ts, "%Y/%m/%d %H:%M:%S")) + (float("0." + frac) if frac else 0.0)
                rows.append((ts, float(parts[2]), float(parts[3]), parts[5:]))
            except (ValueError, IndexError):
                continue
        os.unlink(self.file.name)
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05]
        use = inside or rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in use for n, v in zip(names, r[3][1:]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use), "samples_in_region": len(inside)}


# ---------------------------------------------------------------------------------------------

def oracle_rate(orc, key, data_blocks: np.ndarray, cores: int, target_s: float, max_blocks: int) -> tuple[float, int]:
    """Calibrate: oracle blocks per second (encrypt) on `cores` threads."""
    probe = min(max_blocks, max(cores * 256, 4096))
    t = time.perf_counter()
    orc.encrypt_blocks(key, data_blocks[: probe * 16], threads=cores)
    dt = time.perf_counter() - t
    rate = probe / max(dt, 1e-6)
    return rate, int(min(max_blocks, max(probe, rate * target_s / 2)))


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, timed on the host cores."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import oracle

    orc = oracle.oracle()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(SEED)
    key = rng.integers(0, 256, 16, dtype=np.uint8)
    # bounded sample of the same workload: the first S blocks of the seed-1 buffer (drawn
    # in the same order as workloads.plain, so the blocks are the benchmark's own)
    budget_s = 150.0
    rate, _ = oracle_rate(orc, key, rng.integers(0, 256, 16 * 8192, dtype=np.uint8), cores, 1.0, 8192)
    per_step = int(max(1024, min(NBLOCKS, rate * budget_s / max(1, args.steps + args.warmup) / 2)))
    data = workloads.plain(SEED, per_step).data
    for _ in range(args.warmup):
        ct = orc.encrypt_blocks(key, data, threads=cores)
        orc.decrypt_blocks(key, ct, threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        ct = orc.encrypt_blocks(key, data, threads=cores)
        pt = orc.decrypt_blocks(key, ct, threads=cores)
    dt = time.perf_counter() - t
    assert (pt == data).all()
    value = 2 * per_step * 16 * args.steps / dt / 1e9
    sample = f"first {per_step} blocks of the seed-1 1 GiB workload per step, encrypt+decrypt"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_blocks_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def read_profile_traffic() -> float | None:
    """DRAM bytes per launch of the encryption kernel, from the committed ncu summary (the
    line `traffic_bytes_per_launch: <n>` of the committed ncu summary of the encryption kernel)."""
    f = ROOT / "profiles" / "tt_kernel_aes128_256MiB.md"
    if not f.exists():
        return None
    for line in f.read_text().splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            try:
                return float(line.split(":", 1)[1].strip().split()[0])
            except ValueError:
                return None
    return None


def run_ours(args):
    import torch

    import paper_1506_08503_gb300 as aes

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if dist is not None:
            dist.barrier()

    n = args.nblocks
    # weak scaling: every rank processes its own 1 GiB batch (rank 0 holds the seed-1 data)
    w = workloads.plain(SEED + 1000 * rank, n)
    x = torch.from_numpy(w.data).to(dev)
    ct = torch.empty_like(x)
    pt = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    key = w.key.tobytes()
    lib = aes.lib()
    import ctypes

    ks = aes.aes_key_schedule()
    kbuf = (ctypes.c_uint8 * 16).from_buffer_copy(key)
    impl = {"auto": 0, "ttable": 1, "bitslice": 2}[args.kernel]
    xp, cp, pp = x.data_ptr(), ct.data_ptr(), pt.data_ptr()

    def step(events=None):
        st = lib.aes_key_expand(kbuf, 128, ctypes.byref(ks))
        if events:
            events[0].record(stream)
        st |= lib.aes_crypt_blocks(ctypes.byref(ks), None, xp, cp, n, 0, impl, sptr)
        if events:
            events[1].record(stream)
        st |= lib.aes_crypt_blocks(ctypes.byref(ks), None, cp, pp, n, 1, impl, sptr)
        if events:
            events[2].record(stream)
        if st != 0:
            raise RuntimeError(aes.aes_last_error())

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if not torch.equal(pt, x):
        raise RuntimeError("round trip failed: decrypt(encrypt(x)) != x")

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    barrier()
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    enc_ms = [e[0].elapsed_time(e[1]) for e in evs]
    dec_ms = [e[1].elapsed_time(e[2]) for e in evs]
    if not torch.equal(pt, x):
        raise RuntimeError("round trip failed after the timed region")

    ms_max = ms
    if dist is not None:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    bytes_per_step_rank = 2 * n * 16
    value = bytes_per_step_rank * world * args.steps / (ms_max / 1e3) / 1e9

    # ---- e2e through the host-buffer entry point -------------------------------------------
    e2e = None
    if not args.no_e2e:
        hx = torch.from_numpy(w.data).pin_memory()
        hc = torch.empty_like(hx).pin_memory()
        hp = torch.empty_like(hx).pin_memory()

        def host_step():
            st = lib.aes_key_expand(kbuf, 128, ctypes.byref(ks))
            st |= lib.aes_crypt_host(ctypes.byref(ks), None, hx.data_ptr(), hc.data_ptr(), n, 0, impl, sptr)
            st |= lib.aes_crypt_host(ctypes.byref(ks), None, hc.data_ptr(), hp.data_ptr(), n, 1, impl, sptr)
            if st != 0:
                raise RuntimeError(aes.aes_last_error())

        e2e_steps = max(1, min(args.steps, 20))
        for _ in range(max(1, min(args.warmup, 3))):
            host_step()
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            host_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        if dist is not None:
            tt = torch.tensor([dt], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            dt = float(tt.item())
        if not torch.equal(hp, hx):
            raise RuntimeError("host-buffer round trip failed")
        e2e = {"value": bytes_per_step_rank * world * e2e_steps / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * 16, "d2h_bytes_per_step": 2 * n * 16,
               "steps": e2e_steps, "api": "aes_crypt_host (pinned host buffers)"}
        del hx, hc, hp

    # ---- roofline of the dominant kernel -----------------------------------------------------
    enc_avg, dec_avg = statistics.mean(enc_ms), statistics.mean(dec_ms)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = roofline_peak_gbs(sms, SM_MAX_MHZ_NOMINAL)
    dom_ms = max(enc_avg, dec_avg)
    dom = "encrypt" if enc_avg >= dec_avg else "decrypt"
    achieved = n * 16 / (dom_ms / 1e3) / 1e9
    traffic = read_profile_traffic() if args.kernel in ("auto", "ttable") and n == NBLOCKS else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": f"tt_kernel<10,{dom}>" if args.kernel != "bitslice" else f"bitslice<10,{dom}>",
                "peak_source": f"derived: {sms} SMs x {SM_MAX_MHZ_NOMINAL:.0f} MHz x {blocks_per_sm_clock():.4f} blocks/SM-clock x 16 B",
                "enc_gbs": n * 16 / (enc_avg / 1e3) / 1e9, "dec_gbs": n * 16 / (dec_avg / 1e3) / 1e9,
                "hbm_term_gbs": 6774.2 / 2}

    # ---- CPU oracle baseline (rank 0, N = 1 only) ---------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        orc = oracle.oracle()
        cores = os.cpu_count() or 1
        _, s = oracle_rate(orc, w.key, w.data, cores, args.cpu_seconds, n)
        sample = w.data[: s * 16]
        t = time.perf_counter()
        oct_ = orc.encrypt_blocks(w.key, sample, threads=cores)
        opt = orc.decrypt_blocks(w.key, oct_, threads=cores)
        dt = time.perf_counter() - t
        gpu_ct = ct[: s * 16].cpu().numpy()
        cpu = {"value": 2 * s * 16 / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {s} blocks of the 1 GiB seed-1 workload, encrypt then decrypt",
               "seconds": dt, "gpu_matches_oracle_on_sample": bool((gpu_ct == oct_).all() and (opt == sample).all())}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nblocks_per_rank": n, "key_bits": 128, "mode": "ECB (IV = 0)",
                       "kernel": args.kernel, "l2": "inputs (1 GiB) larger than L2 (129 MB); no flush"},
            "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clk, "roofline": roofline,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
