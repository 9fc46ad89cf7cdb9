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
import gc
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

from paper_1506_08503_gb300 import sharding, workloads  # noqa: E402

METRIC = "AES-128 encrypt+decrypt throughput, many independent 16-byte blocks"
UNIT = "GB/s"
WORKLOAD = "aes128-enc+dec-1GiB-2^26-blocks-seed1"
NBLOCKS = 1 << 26
SEED = 1

# On-chip integer roofline: per SM and clock the GB300 issues
# 64 lanes of integer ALU work (LOP3/PRMT/SHF/IADD, measured) and 32 lanes of shared-memory
# loads.  A table-lookup AES-128 block needs at least 160 lookups and 240 ALU operations; a
# gate-level (bitsliced) block at least 356.25 ALU lane-operations (22,800 two-input gates,
# two per LOP3, 32 blocks per lane).  Filling the LDS pipe with lookups and the ALU pipe's
# remainder with gates gives 0.2449 blocks per SM-clock.
ALU_LANES, LDS_LANES = 64.0, 32.0
TT_LDS, TT_ALU, BS_ALU = 160.0, 240.0, 22800.0 / 64.0
SM_COUNT_NOMINAL, SM_MAX_MHZ_NOMINAL = 152, 2070.0
# The bitsliced kernel's own instruction count on the integer ALU pipe per AES-128 block (LOP3 +
# PRMT + SHF, from ncu's per-opcode counts at 2^24 blocks, profiles/bs_kernel_aes128_256MiB.md):
# the ceiling of this circuit and layout, beside the gate-level bound of the best circuits.
BS_KERNEL_ALU = {"encrypt": 511.5 + 16.0 + 12.0, "decrypt": 567.8 + 16.0 + 12.0}


def blocks_per_sm_clock() -> float:
    t = min(LDS_LANES / TT_LDS, ALU_LANES / TT_ALU)
    b = max(0.0, (ALU_LANES - TT_ALU * t) / BS_ALU)
    return t + b


def roofline_peak_gbs(sms: int, mhz: float) -> float:
    return blocks_per_sm_clock() * sms * mhz * 1e6 * 16 / 1e9


def lds_path_bound_gbs(sms: int, mhz: float, wavefronts_per_block: float) -> float:
    """A table-lookup kernel's own ceiling: one 128-byte shared-memory wavefront per SM-clock,
    `wavefronts_per_block` of them per 16-byte block (lookups plus the block's load and store,
    1/8 wavefront each)."""
    return sms * mhz * 1e6 / wavefronts_per_block * 16 / 1e9


def ttable_wavefronts(nr: int) -> float:
    """16 conflict-free lookups (half a wavefront) per round, plus the block's load and store."""
    return nr / 2.0 + 0.25


# GCM adds 2.5 wavefronts of GHASH lookups per block to the counter-mode data pass
GCM_WAVEFRONTS = ttable_wavefronts(10) + 2.5


def hbm_peak_gbs() -> float:
    """Measured copy bandwidth (read + write bytes per second) of the GB300s."""
    f = ROOT / "MEASURED_PEAKS.json"
    try:
        return float(json.loads(f.read_text())["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6774.2  # the same measurement as recorded when the file is absent


def logic_bound_gbs(sms: int, mhz: float, lane_ops_per_block: float = BS_ALU) -> float:
    """The gate-level bound: the ALU pipe's 64 lanes per SM-clock over the lane-operations a
    bitsliced block needs (356.25 for AES-128 at two gates per LOP3)."""
    return sms * mhz * 1e6 * ALU_LANES / lane_ops_per_block * 16 / 1e9


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
    p.add_argument("--no-batched", action="store_true", help="skip the 4096-message batched measurement")
    p.add_argument("--no-bitsliced", action="store_true", help="skip the bitsliced kernel's 1 GiB measurement")
    p.add_argument("--tt-shape", default=None,
                   help="T,U: set the AUTO kernel to the T-table kernel with this CTA size and blocks per "
                        "thread instead of running the launch tuner (for profiling)")
    p.add_argument("--batched-shape", default=None,
                   help="T,U: run the batched measurement at this CTA size and blocks per lane instead of "
                        "autotuning (the tuner's timings are meaningless under a profiler)")
    p.add_argument("--no-served", action="store_true", help="skip the served (request server) measurement")
    p.add_argument("--served-requests", type=int, default=10000, help="requests per offered rate")
    p.add_argument("--no-cbc", action="store_true", help="skip the multi-block CBC measurement")
    p.add_argument("--no-followons", action="store_true", help="skip the counter-mode and column-scan measurements")
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

def openssl_ecb(key: np.ndarray, data: np.ndarray, cores: int, seconds: float, check: np.ndarray | None):
    """Context, not a target: AES-128 ECB encryption of `data` through the host's OpenSSL
    (libcrypto's EVP interface, which uses the CPU's AES instructions), the kind of CPU library
    the paper compares against (Section IV), on `cores` threads for about `seconds`.  `check`,
    if given, is the expected ciphertext of the first blocks.  None when no libcrypto loads."""
    import ctypes
    import ctypes.util
    import threading

    lib = None
    for name in [ctypes.util.find_library("crypto"), "libcrypto.so.3", "libcrypto.so.1.1", "libcrypto.so"]:
        if not name:
            continue
        try:
            lib = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if lib is None:
        return None
    vp, ip = ctypes.c_void_p, ctypes.c_int
    lib.EVP_CIPHER_CTX_new.restype = vp
    lib.EVP_aes_128_ecb.restype = vp
    lib.EVP_EncryptInit_ex.argtypes = [vp, vp, vp, vp, vp]
    lib.EVP_CIPHER_CTX_set_padding.argtypes = [vp, ip]
    lib.EVP_EncryptUpdate.argtypes = [vp, vp, ctypes.POINTER(ip), vp, ip]
    lib.EVP_CIPHER_CTX_free.argtypes = [vp]
    kb = np.ascontiguousarray(key, dtype=np.uint8)
    out = np.empty_like(data)
    n = data.size // 16
    bounds = [16 * (n * i // cores) for i in range(cores + 1)]
    done = [0] * cores
    stop = time.perf_counter() + seconds
    errors = []

    def work(i):
        ctx = lib.EVP_CIPHER_CTX_new()
        try:
            if not ctx or lib.EVP_EncryptInit_ex(ctx, lib.EVP_aes_128_ecb(), None, kb.ctypes.data, None) != 1:
                errors.append("EVP_EncryptInit_ex")
                return
            lib.EVP_CIPHER_CTX_set_padding(ctx, 0)
            outl = ip(0)
            lo, hi = bounds[i], bounds[i + 1]
            while True:
                for a in range(lo, hi, 1 << 26):  # 64 MiB per call
                    b = min(hi, a + (1 << 26))
                    if lib.EVP_EncryptUpdate(ctx, out.ctypes.data + a, ctypes.byref(outl), data.ctypes.data + a,
                                             b - a) != 1:
                        errors.append("EVP_EncryptUpdate")
                        return
                    done[i] += b - a
                if time.perf_counter() >= stop:
                    return
        finally:
            if ctx:
                lib.EVP_CIPHER_CTX_free(ctx)

    t = time.perf_counter()
    threads = [threading.Thread(target=work, args=(i,)) for i in range(cores)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    dt = time.perf_counter() - t
    if errors:
        return {"error": errors[0]}
    res = {"encrypt_gbs": sum(done) / dt / 1e9, "threads": cores, "bytes": int(sum(done)), "seconds": dt,
           "library": "OpenSSL libcrypto EVP aes-128-ecb", "role": "context (a CPU library comparator), not a target"}
    if check is not None:
        res["matches_gpu_on_first_blocks"] = bool(np.array_equal(out[: check.size], check))
    return res


def oracle_rate(orc, key, data_blocks: np.ndarray, cores: int, target_s: float, max_blocks: int) -> tuple[float, int]:
    """Calibrate: oracle blocks per second (encrypt) on `cores` threads."""
    # large enough that thread start-up does not dominate (a 4096-block probe on 16 cores
    # underestimated the rate about twofold, so samples came out at half their target time)
    probe = min(max_blocks, max(cores * 4096, 16384))
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


def read_profile() -> dict:
    """From the committed ncu summary of the T-table kernel: the (threads, blocks per thread)
    shape it was taken on (`profiled_shape:`), DRAM bytes per 2^26-block launch per direction
    (`traffic_bytes_per_launch:` for encryption, `..._decrypt:`) and per-direction counters
    (`ncu_encrypt:` / `ncu_decrypt:`, key=value pairs)."""
    f = ROOT / "profiles" / "tt_kernel_aes128_256MiB.md"
    out = {"shape": None, "traffic": {}, "ncu": {}, "source": f"profiles/{f.name}"}
    if not f.exists():
        return out
    for line in f.read_text().splitlines():
        key, _, rest = line.partition(":")
        if key == "profiled_shape":
            t, u = rest.split()[0].split(",")
            out["shape"] = (int(t), int(u))
        elif key == "traffic_bytes_per_launch":
            out["traffic"]["encrypt"] = float(rest.split()[0])
        elif key == "traffic_bytes_per_launch_decrypt":
            out["traffic"]["decrypt"] = float(rest.split()[0])
        elif key in ("ncu_encrypt", "ncu_decrypt"):
            out["ncu"][key[4:]] = {k: float(v) for k, v in (kv.split("=") for kv in rest.split())}
    return out


def measure_bitsliced(aes, torch, dev, x, n: int, key: bytes, sms: int, gpu: int = 0) -> dict:
    """The constant-time bitsliced kernel on the benchmark's 1 GiB buffer (AES-128, 40 launches
    per direction after 2 warm-ups, CUDA events), against its gate-level bound, with the SM
    clocks sampled over its own timed region (the kernel keeps the integer pipe busier than
    the T-table kernel does, so the power cap can lower the clock here and not there)."""
    stream = torch.cuda.current_stream()
    ks = aes.aes_key_expand(key)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    out = {}
    clocks = Clocks(gpu)
    clocks.start()
    clocks.mark("t0")
    for d, src, dst in (("encrypt", x, y), ("decrypt", y, z)):
        for _ in range(2):
            aes.aes_crypt_blocks(ks, None, src.data_ptr(), dst.data_ptr(), n, d, "bitslice")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(40):
            aes.aes_crypt_blocks(ks, None, src.data_ptr(), dst.data_ptr(), n, d, "bitslice")
        e1.record(stream)
        torch.cuda.synchronize()
        out[d + "_gbs"] = n * 16 / (e0.elapsed_time(e1) / 40 / 1e3) / 1e9
    clocks.mark("t1")
    out["clocks"] = clocks.stop()
    if not torch.equal(z, x):
        raise RuntimeError("bitsliced round trip failed")
    bound = logic_bound_gbs(sms, SM_MAX_MHZ_NOMINAL)
    out.update({"logic_bound_gbs": bound, "encrypt_frac": out["encrypt_gbs"] / bound,
                "decrypt_frac": out["decrypt_gbs"] / bound,
                "bound_source": f"{sms} SMs x {SM_MAX_MHZ_NOMINAL:.0f} MHz x {ALU_LANES:.0f} lanes / "
                                f"{BS_ALU} lane-ops per block x 16 B"})
    for d in ("encrypt", "decrypt"):
        kb = logic_bound_gbs(sms, SM_MAX_MHZ_NOMINAL, BS_KERNEL_ALU[d])
        out[f"{d}_kernel_alu_bound_gbs"] = kb
        out[f"{d}_frac_of_kernel_alu_bound"] = out[f"{d}_gbs"] / kb
    out["kernel_alu_bound_source"] = (f"{sms} SMs x {SM_MAX_MHZ_NOMINAL:.0f} MHz x {ALU_LANES:.0f} lanes / the kernel's "
                                      f"ALU-pipe instructions per block (ncu: {BS_KERNEL_ALU['encrypt']} encrypt, "
                                      f"{BS_KERNEL_ALU['decrypt']} decrypt) x 16 B")
    del y, z
    return out


def summary_of(line: dict, sms: int) -> dict:
    """The headline figures of every configuration in one small object, printed last on the line."""
    mhz = SM_MAX_MHZ_NOMINAL
    r = line["roofline"]
    s = {"plain_1GiB": {"gbs": line["value"], "enc_gbs": r["enc_gbs"], "dec_gbs": r["dec_gbs"], "frac": r["frac"],
                        "frac_of_lds_path_bound": r["frac_of_lds_path_bound"]},
         "e2e_gbs": (line.get("e2e") or {}).get("value")}
    bs = line.get("bitsliced")
    if bs:
        s["bitsliced_1GiB"] = {k: bs[k] for k in ("encrypt_gbs", "decrypt_gbs", "encrypt_frac", "decrypt_frac",
                                                 "logic_bound_gbs", "encrypt_frac_of_kernel_alu_bound",
                                                 "decrypt_frac_of_kernel_alu_bound")}
        s["bitsliced_1GiB"]["sm_mhz"] = bs["clocks"].get("sm_mhz")
    b = line.get("batched")
    if b:
        s["batched_4096_msgs"] = {"gbs": b["value"], "vs_plain_kernel": b["vs_plain_kernel"],
                                  "vs_plain_kernel_same_bytes": b["vs_plain_kernel_same_bytes"]}
        if b.get("with_ivs"):
            s["batched_4096_msgs"]["with_ivs_gbs"] = b["with_ivs"]["value"]
    f = line.get("followons")
    if f:
        b10, b14 = (lds_path_bound_gbs(sms, mhz, ttable_wavefronts(nr)) for nr in (10, 14))
        sen = f["sensor_1e7_records"]
        s["sensor_1e7_records"] = {
            "aes128_enc_gbs": sen["aes128_encrypt_gbs"], "aes128_frac": sen["aes128_encrypt_gbs"] / b10,
            "aes256_enc_gbs": sen["aes256_encrypt_gbs"], "aes256_frac": sen["aes256_encrypt_gbs"] / b14,
            "bounds_gbs": {"aes128": b10, "aes256": b14}}
        gb = lds_path_bound_gbs(sms, mhz, GCM_WAVEFRONTS)
        s["ctr_1GiB"] = {"gbs": f["ctr_1GiB_gbs"], "frac": f["ctr_1GiB_gbs"] / b10, "bound_gbs": b10}
        s["gcm_1GiB"] = {"enc_gbs": f["gcm_1GiB_encrypt_gbs"], "dec_gbs": f["gcm_1GiB_decrypt_gbs"],
                         "frac": f["gcm_1GiB_encrypt_gbs"] / gb, "bound_gbs": gb}
        s["scan_1e7_records"] = {"gbs": f["scan_1e7_records_gbs"], "frac": f["scan_frac_of_measured_copy_bw"]}
        sm = f.get("small_4096_blocks")
        if sm:
            s["small_4096_blocks_us"] = {k: sm[k] for k in ("encrypt_us_median", "encrypt_graph_replay_us_median",
                                                           "decrypt_us_median", "decrypt_graph_replay_us_median")}
    c = line.get("cbc")
    if c:
        s["cbc"] = [{"msgs": row["messages"], "blocks": row["blocks_per_message"], "enc_gbs": row["encrypt_gbs"],
                     "dec_gbs": row["decrypt_gbs"]} for row in c["rows"] + [c["varying_lengths_own_keys"]]]
    v = line.get("served")
    if v:
        cl = v["closed_loop"]
        s["served"] = {"closed_loop": {k: cl[k] for k in ("gbps", "gbps_from_first_launch",
                                                          "vs_plain_kernel_same_rounds_wall",
                                                          "vs_plain_kernel_same_rounds", "p50_us", "p99_us")},
                       "rates": [{"rate": e["offered_rate"], "p50_us": e["p50_us"], "p99_us": e["p99_us"]}
                                 for e in v["rates"]]}
    return s


def measure_batched(aes, torch, dev, steps: int, plain_gbs: float, fixed_shape=None) -> dict:
    """4096 messages, lognormal lengths (median 4 KiB, sigma 1.5), one AES-128 key each (seed 3),
    encrypted in one autotuned persistent launch per step.  Four copies of the 52.6 MB workload
    sit at different places in device memory and the steps cycle through them back to back, so
    every batch reads data that three batches (over 300 MB of traffic) have pushed out of L2;
    the host prepares batch k+1 while the GPU runs batch k, as a pipelined caller would."""
    m = workloads.batched_messages(3)
    total = int(m.lengths.sum())
    copies = 4
    msgs = np.zeros(len(m.lengths), dtype=aes.msg_dtype())
    msgs["key_idx"] = np.arange(len(m.lengths))
    msgs["offset"], msgs["length"] = m.offsets, m.lengths
    stream = torch.cuda.current_stream()
    with aes.KeyPool(len(m.keys)) as pool:
        pool.load_keys(0, m.keys, 128)
        x = torch.from_numpy(np.tile(m.data, copies)).to(dev)
        y = torch.empty_like(x)
        with aes.Batch(pool, len(m.lengths)) as b:
            if fixed_shape:
                b.set_shape(*fixed_shape)
                shape = tuple(fixed_shape)
            else:
                shape = b.autotune(msgs, x.data_ptr(), y.data_ptr(), total)
            ptrs = [(x.data_ptr() + k * total, y.data_ptr() + k * total) for k in range(copies)]
            for k in range(2 * copies):
                b.run(msgs, *ptrs[k % copies], total)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(steps):
                b.run(msgs, *ptrs[k % copies], total)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            # the plain single-key kernel on the same bytes, same copies and back-to-back timing
            ks0 = aes.aes_key_expand(m.keys[0].tobytes())
            e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e2.record(stream)
            for k in range(steps):
                aes.aes_crypt_blocks(ks0, None, ptrs[k % copies][0], ptrs[k % copies][1], total // 16, "encrypt",
                                     "ttable")
            e3.record(stream)
            torch.cuda.synchronize()
            plain_same = total / (e2.elapsed_time(e3) / steps / 1e3) / 1e9
            # host cost of one run with the GPU idle
            import time as _t
            t = _t.perf_counter()
            b.run(msgs, *ptrs[0], total)
            host_us = (_t.perf_counter() - t) * 1e6
            torch.cuda.synchronize()
    gbs = total / (ms / 1e3) / 1e9
    return {"workload": "4096 msgs, lognormal(median 4 KiB, sigma 1.5) in [16 B, 16 MiB], own AES-128 key each, seed 3",
            "bytes": total, "value": gbs, "unit": UNIT, "ms_per_batch": ms, "host_us_per_run": host_us,
            "shape": {"threads": shape[0], "blocks_per_lane": shape[1]},
            "vs_plain_kernel": gbs / plain_gbs if plain_gbs else None,
            "plain_kernel_same_bytes_gbs": plain_same, "vs_plain_kernel_same_bytes": gbs / plain_same,
            "l2": "4 copies of the workload cycled (each batch's input last touched >300 MB of traffic ago)",
            "launch": "aes_batch_run back to back (descriptor upload on a copy stream + CUDA graph replay)"}


def measure_cbc(aes, torch, dev) -> dict:
    """The paper's CBC mode over whole messages (App. A1/A4): 128 messages of growing length
    (the paper's second workload shape) and 2^18 messages of 16 blocks; AES-128, one IV per
    message.  Encryption chains inside each message (one lane per message); decryption is
    block-parallel.  GB/s of message bytes, CUDA events, 5 repetitions after 2 warm-ups."""
    ks = aes.aes_key_expand(bytes(range(16)))
    stream = torch.cuda.current_stream()
    rows = []
    for n, m in ((128, 16), (128, 256), (128, 4096), (1 << 18, 16)):
        x = torch.randint(0, 256, (n, 16 * m), dtype=torch.uint8, device=dev)
        ivs = torch.randint(0, 256, (n, 16), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        entry = {"messages": n, "blocks_per_message": m, "bytes": n * m * 16}
        for d, src, dst in (("encrypt", x, y), ("decrypt", y, z)):
            for _ in range(2):
                aes.cbc(src, ks, ivs, d, out=dst)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                aes.cbc(src, ks, ivs, d, out=dst)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            entry[d + "_gbs"] = n * m * 16 / (ms / 1e3) / 1e9
        if n * m >= 1 << 20:
            # the independent-block kernel on the same bytes (ECB, same key): what the chain
            # and the previous-block read cost
            xf, yf = x.view(-1), y.view(-1)
            for d, fn in (("encrypt", aes.encrypt), ("decrypt", aes.decrypt)):
                for _ in range(2):
                    fn(xf, ks, out=yf)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(5):
                    fn(xf, ks, out=yf)
                e1.record(stream)
                torch.cuda.synchronize()
                entry["ecb_same_bytes_" + d + "_gbs"] = n * m * 16 / (e0.elapsed_time(e1) / 5 / 1e3) / 1e9
        torch.cuda.synchronize()
        if not torch.equal(z, x):
            raise RuntimeError("CBC round trip failed")
        rows.append(entry)
    out = {"mode": "CBC over whole messages, AES-128, one IV per message", "rows": rows}
    # the general form through aes_cbc_batched: 128 messages of lengths 1 .. 4096 blocks
    # (geometric), each with its own AES-128 key and IV
    rng = np.random.default_rng(5)
    n = 128
    lengths = np.resize(np.unique(np.geomspace(1, 4096, n).astype(np.int64)), n) * 16
    offs = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    total = int(lengths.sum())
    msgs = np.zeros(n, dtype=aes.msg_dtype())
    msgs["key_idx"], msgs["offset"], msgs["length"] = np.arange(n), offs, lengths
    ivs = rng.integers(0, 256, (n, 16), dtype=np.uint8)
    with aes.KeyPool(n) as pool:
        pool.load_keys(0, rng.integers(0, 256, (n, 16), dtype=np.uint8), 128)
        x = torch.randint(0, 256, (total,), dtype=torch.uint8, device=dev)
        y, z = torch.empty_like(x), torch.empty_like(x)
        entry = {"messages": n, "blocks_per_message": "1..4096 (geometric)", "bytes": total,
                 "api": "aes_cbc_batched (own key and IV per message)"}
        for d, src, dst in (("encrypt", x, y), ("decrypt", y, z)):
            msgs["dir"] = 0 if d == "encrypt" else 1
            for _ in range(2):
                aes.aes_cbc_batched(pool, msgs, ivs, src.data_ptr(), dst.data_ptr(), total)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                aes.aes_cbc_batched(pool, msgs, ivs, src.data_ptr(), dst.data_ptr(), total)
            e1.record(stream)
            torch.cuda.synchronize()
            entry[d + "_gbs"] = total / (e0.elapsed_time(e1) / 5 / 1e3) / 1e9
        if not torch.equal(z, x):
            raise RuntimeError("batched CBC round trip failed")
        out["varying_lengths_own_keys"] = entry
    return out


def measure_small_latency(aes, torch, dev) -> dict:
    """The oracle-sized case: 4096 blocks (64 KiB, seed 0) encrypted then decrypted, one call at a
    time on an idle GPU; this fits in L2 and is bound by launch latency, so it is reported in
    microseconds (median over 200 calls, CUDA events around each call: through the Python
    binding, and as a replayed CUDA graph of the same call).  AES_IMPL_AUTO takes the small-call
    kernel (tables from global memory); the shared-memory T-table kernel is timed beside it."""
    w = workloads.plain(0, 4096)
    ks = aes.aes_key_expand(w.key.tobytes())
    x = torch.from_numpy(w.data).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    out = {}

    def per_call(fn):
        times = []
        for k in range(210):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= 10:
                times.append(e0.elapsed_time(e1) * 1e3)
        return statistics.median(times)

    for d, src, dst in (("encrypt", x, y), ("decrypt", y, x)):
        for impl, tag in (("auto", ""), ("ttable", "_smem_ttable")):
            call = (lambda s=src, t=dst, dd=d, i=impl:
                    aes.aes_crypt_blocks(ks, None, s.data_ptr(), t.data_ptr(), 4096, dd, i))
            out[d + tag + "_us_median"] = per_call(call)
            # the same call captured once in a CUDA graph and replayed: the device-side latency,
            # without the Python and ctypes path in front of the launch
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                call()
            out[d + tag + "_graph_replay_us_median"] = per_call(g.replay)
            del g
    if not torch.equal(x, torch.from_numpy(w.data).to(dev)):
        raise RuntimeError("4096-block round trip failed")
    out["workload"] = "4096 blocks (64 KiB), AES-128, seed 0"
    return out


def measure_followons(aes, torch, dev, x, n: int, key: bytes) -> dict:
    """Counter mode and GCM over the benchmark's 1 GiB buffer, and an equality scan of a 10^7-record
    encrypted sensor column (160 MB, read once: an HBM-bound kernel, reported against the
    measured copy bandwidth as read bytes per second)."""
    stream = torch.cuda.current_stream()
    ks = aes.aes_key_expand(key)
    y = torch.empty_like(x)
    ctr0 = bytes(range(16))

    def timed(fn, reps):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_ctr = timed(lambda: aes.aes_ctr_crypt(ks, ctr0, x.data_ptr(), y.data_ptr(), n), 10)
    col = workloads.sensor_records(2, 10_000_000)
    # the sensor column itself (10^7 16-byte records, 160 MB) under AES-128 and AES-256
    recs = torch.from_numpy(col.records).to(dev)
    rout = torch.empty_like(recs)
    sensor = {}
    for name, kb in (("aes128", col.key128), ("aes256", col.key256)):
        kss = aes.aes_key_expand(kb.tobytes())
        for d in ("encrypt", "decrypt"):
            ms_s = timed(lambda: aes.aes_crypt_blocks(kss, None, recs.data_ptr(), rout.data_ptr(), 10_000_000, d,
                                                      "ttable"), 10)
            sensor[f"{name}_{d}_gbs"] = 160e6 / (ms_s / 1e3) / 1e9
    del rout
    enc = aes.encrypt(torch.from_numpy(col.records).to(dev), aes.aes_key_expand(col.key128.tobytes()))
    needle = bytes(aes.encrypt(enc[:16].clone(), ks).cpu().numpy())  # any 16 bytes: almost surely absent
    matches = torch.empty(1024, dtype=torch.int64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    ms_scan = timed(lambda: aes.aes_scan_equal(enc.data_ptr(), 10_000_000, needle, matches.data_ptr(), 1024,
                                               count.data_ptr()), 20)
    scan_gbs = 160e6 / (ms_scan / 1e3) / 1e9
    # GCM over the same 1 GiB (16 KiB of AAD), each call = set-up, data pass and combine kernels
    iv = bytes(range(12))
    aad = torch.randint(0, 256, (16384,), dtype=torch.uint8, device=dev)
    work = torch.empty(aes.aes_gcm_workspace_bytes(), dtype=torch.uint8, device=dev)
    tag = torch.empty(16, dtype=torch.uint8, device=dev)

    def gcm_call(d, m):
        aes.aes_gcm_crypt(ks, iv, aad.data_ptr(), aad.numel(), x.data_ptr(), y.data_ptr(), m * 16, d, tag.data_ptr(),
                          work.data_ptr(), work.numel())

    ms_gcm_enc = timed(lambda: gcm_call("encrypt", n), 10)
    ms_gcm_dec = timed(lambda: gcm_call("decrypt", n), 10)
    us_gcm_small = timed(lambda: gcm_call("encrypt", 4096), 50) * 1e3
    return {"ctr_1GiB_gbs": n * 16 / (ms_ctr / 1e3) / 1e9,
            "gcm_1GiB_encrypt_gbs": n * 16 / (ms_gcm_enc / 1e3) / 1e9,
            "gcm_1GiB_decrypt_gbs": n * 16 / (ms_gcm_dec / 1e3) / 1e9,
            "gcm_4096_blocks_us": us_gcm_small,
            "gcm_note": "AES-128-GCM, 96-bit IV, 16 KiB AAD; one kernel launch per call after a 4-byte memset of the combine ticket",
            "sensor_1e7_records": sensor,
            "scan_1e7_records_gbs": scan_gbs, "scan_ms": ms_scan,
            "scan_frac_of_measured_copy_bw": scan_gbs / 6774.2,
            "note": "scan reads 16 B per record once; L2 (129 MB) holds part of the 160 MB column between repetitions"}


def measure_served(aes, torch, dev, nreq: int, plain_gbs: float, closed_n: int = 1_000_000) -> dict:
    """The request server under Poisson arrivals (seed 4): 50/50 encrypt/decrypt, sizes
    lognormal (median 4 KiB, sigma 1.5) in [64 B, 64 MiB], keys from a resident pool of 1024
    (512 AES-128, 512 AES-256), payloads resident in device memory.  Offered rates 1k, 3k,
    10k, 30k and 100k requests/s (nreq requests each, 10 * nreq at 100k/s: one to ten seconds
    of arrivals per rate), then a closed loop for saturation: the configuration's 10^6 requests
    handed to the server as fast as the client can (calls of 8192 requests, back to back), over
    the server's own window from the first submission to the last completion; one warm-up
    repetition (reported apart), then the median of three."""
    import time as _t

    out = {"workload": "Poisson arrivals, 50/50 enc/dec, lognormal(median 4 KiB, sigma 1.5) in [64 B, 64 MiB], "
                       "1024-key pool (half AES-128, half AES-256), device-resident payloads, seed 4",
           "requests_per_rate": {"1k-30k req/s": nreq, "100k req/s": 10 * nreq}, "closed_loop_requests": closed_n,
           "rates": []}
    w0 = workloads.served_requests(4, 1, 1.0)
    pool = aes.KeyPool(len(w0.pool_keys))
    pool.load_keys(0, np.stack(w0.pool_keys[:512]), 128)
    pool.load_keys(512, np.stack(w0.pool_keys[512:]), 256)
    # the worker keeps polling for 2 ms after its last request or batch (one host core), so that
    # requests arriving at least every 2 ms find it awake instead of paying a thread wake-up
    srv = aes.Server(pool, hbm_budget=1 << 30, max_inflight=1 << 21, nstreams=4, max_batch=8192,
                     queue_capacity=1 << 21, linger_us=2000)
    out["server_cfg"] = {"nstreams": 4, "max_batch": 8192, "hbm_budget": 1 << 30, "linger_us": 2000}
    try:
        for rate in (1000.0, 3000.0, 10000.0, 30000.0, 100000.0, None):
            count = closed_n if rate is None else 10 * nreq if rate >= 1e5 else nreq
            w = workloads.served_requests(4, count, rate or 1e9)
            offs = np.concatenate([[0], np.cumsum(w.lengths)[:-1]]).astype(np.int64)
            total = int(w.lengths.sum())
            src = torch.randint(0, 256, (total,), dtype=torch.uint8, device=dev)
            dst = torch.empty_like(src)
            torch.cuda.synchronize()
            sp, dp = src.data_ptr(), dst.data_ptr()
            srv.reset_stats()
            tickets = []
            t0 = _t.perf_counter()
            if rate:
                # the client's own pauses would show as bursts in the offered load: no Python
                # garbage collection while it submits (the server's threads are native)
                arrivals, kidx, dirs, lens = (w.arrival_s.tolist(), w.key_idx.tolist(), w.dirs.tolist(),
                                              w.lengths.tolist())
                offl = offs.tolist()
                gc.disable()
                try:
                    for i in range(len(lens)):
                        target = t0 + arrivals[i]
                        while _t.perf_counter() < target:
                            pass
                        o = offl[i]
                        tickets.append(srv.submit(kidx[i], dirs[i], sp + o, dp + o, lens[i], True, True))
                finally:
                    gc.enable()
            else:  # closed loop: the whole workload handed over as fast as the client can, the
                # server batches what it finds.  The client submits in calls of 8192 requests
                # (each all or nothing), back to back, and waits on the server's completion count;
                # one warm-up repetition, then three, the median one reported (the loop leans on
                # host threads)
                reqs = np.zeros(len(w.lengths), dtype=aes.request_dtype())
                reqs["key_idx"], reqs["dir"], reqs["length"] = w.key_idx, w.dirs, w.lengths
                reqs["src"], reqs["dst"] = sp + offs, dp + offs
                reqs["src_on_device"], reqs["dst_on_device"] = 1, 1
                chunk = 8192
                reps = []
                for _ in range(4):
                    srv.reset_stats()
                    t0 = _t.perf_counter()
                    tickets = [srv.submit_many(reqs[c:c + chunk]) for c in range(0, len(reqs), chunk)]
                    while srv.stats()["completed"] + srv.stats()["failed"] < len(reqs):
                        _t.sleep(0.0005)
                    dt = _t.perf_counter() - t0
                    st = srv.stats()
                    tickets = np.concatenate(tickets).tolist()
                    states = [srv.poll(t) for t in tickets]  # releases the tickets (all finished)
                    reps.append((st, states, dt))
                out["closed_loop_warmup_gbps"] = reps[0][0]["gbps"]
                reps = sorted(reps[1:], key=lambda r: r[0]["gbps"])
                st, states, dt = reps[1]
                out["closed_loop_repetitions_gbps"] = [r[0]["gbps"] for r in reps]
                out["closed_loop_submission"] = f"calls of {chunk} requests, back to back"
            if rate:
                states = [srv.poll(t) for t in tickets]
                st = srv.stats()
            # completed requests over the server's own window (first submit to last completion),
            # the same window as its gbps
            window_s = st["bytes_completed"] / (st["gbps"] * 1e9) if st["gbps"] > 0 else float("nan")
            entry = {"offered_rate": rate if rate else "closed-loop", "requests": len(tickets),
                     "achieved_rate": st["completed"] / window_s if st["gbps"] > 0 else None,
                     "window": "server clock, first submit to last completion (achieved_rate and gbps)",
                     "p50_us": st["p50_us"], "p99_us": st["p99_us"], "max_us": st["max_us"], "gbps": st["gbps"],
                     "gbps_from_first_launch": st["gbps_from_first_launch"],
                     "mean_batch": st["mean_batch"], "launches": st["launches"],
                     "failed": int(sum(1 for x in states if x != aes.AES_REQ_DONE)), "bytes": total}
            if rate is None:
                # the mix carries 14-round AES-256 requests: compare also against the plain
                # kernel's rate scaled to the byte-weighted mean round count of this workload
                rounds = np.where(w.key_idx < 512, 10.0, 14.0)
                mean_rounds = float((rounds * w.lengths).sum() / w.lengths.sum())
                g = st["gbps_from_first_launch"]
                entry["vs_plain_kernel"] = g / plain_gbs if plain_gbs else None
                entry["mean_rounds_by_bytes"] = mean_rounds
                entry["vs_plain_kernel_same_rounds"] = g / (plain_gbs * 10.0 / mean_rounds) if plain_gbs else None
                entry["vs_plain_kernel_same_rounds_wall"] = (st["gbps"] / (plain_gbs * 10.0 / mean_rounds)
                                                             if plain_gbs else None)
                out["closed_loop"] = entry
            else:
                out["rates"].append(entry)
            del src, dst
        # the same mix end to end: payloads in pinned host memory, staged through the server's
        # HBM arena (bounded by the host link, about 165 GB/s each way when both directions run)
        w = workloads.served_requests(4, 8 * nreq, 1e9)
        offs = np.concatenate([[0], np.cumsum(w.lengths)[:-1]]).astype(np.int64)
        total = int(w.lengths.sum())
        hsrc = torch.randint(0, 256, (total,), dtype=torch.uint8).pin_memory()
        hdst = torch.empty_like(hsrc).pin_memory()
        reqs = np.zeros(len(w.lengths), dtype=aes.request_dtype())
        reqs["key_idx"], reqs["dir"], reqs["length"] = w.key_idx, w.dirs, w.lengths
        reqs["src"], reqs["dst"] = hsrc.data_ptr() + offs, hdst.data_ptr() + offs
        reqs["src_on_device"], reqs["dst_on_device"] = 0, 0
        srv.reset_stats()
        t0 = _t.perf_counter()
        tickets = srv.submit_many(reqs).tolist()
        states = [srv.poll(t) for t in tickets]
        st = srv.stats()
        out["closed_loop_host_payloads"] = {
            "requests": len(tickets), "bytes": total, "gbps": st["gbps"], "p50_us": st["p50_us"], "p99_us": st["p99_us"],
            "mean_batch": st["mean_batch"], "launches": st["launches"],
            "seconds": _t.perf_counter() - t0,
            "failed": int(sum(1 for x in states if x != aes.AES_REQ_DONE)),
            "h2d_bytes": total, "d2h_bytes": total}
        del hsrc, hdst
    finally:
        srv.close()
        pool.close()
    return out


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
    w = workloads.plain(sharding.weak_scaling_seed(SEED, rank), n)
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

    ks0 = aes.aes_key_expand(key)

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

    # the launch tuner picks the AUTO kernel (T-table shapes and the bitsliced kernel), untimed
    tuned = None
    if args.kernel == "auto" and args.tt_shape:
        t_, u_ = (int(v) for v in args.tt_shape.split(","))
        for d in ("encrypt", "decrypt"):
            aes.aes_set_auto_choice(d, 10, "ttable", t_, u_)
        tuned = {d: {"impl": "ttable", "threads": t_, "blocks_per_thread": u_, "set_by": "--tt-shape"}
                 for d in ("encrypt", "decrypt")}
    elif args.kernel == "auto":
        tuned = {d: aes.aes_autotune_blocks(ks0, xp, cp if d == "encrypt" else pp, n, d) for d in ("encrypt", "decrypt")}
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

    ms_max = sharding.max_over_ranks(ms, dev)
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
        dt = sharding.max_over_ranks(dt, dev)
        if not torch.equal(hp, hx):
            raise RuntimeError("host-buffer round trip failed")
        e2e = {"value": bytes_per_step_rank * world * e2e_steps / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * 16, "d2h_bytes_per_step": 2 * n * 16,
               "steps": e2e_steps, "api": "aes_crypt_host (pinned host buffers, read and written by the kernel over the host link where the device allows it, else a copy pipeline)"}
        del hx, hc, hp

    # ---- roofline of the dominant kernel -----------------------------------------------------
    enc_avg, dec_avg = statistics.mean(enc_ms), statistics.mean(dec_ms)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = roofline_peak_gbs(sms, SM_MAX_MHZ_NOMINAL)
    dom_ms = max(enc_avg, dec_avg)
    dom = "encrypt" if enc_avg >= dec_avg else "decrypt"
    achieved = n * 16 / (dom_ms / 1e3) / 1e9
    # the committed ncu traffic figure holds only for the shape it was taken on
    shape = tuned[dom] if tuned else {"impl": args.kernel if args.kernel != "auto" else "ttable", "threads": 512,
                                      "blocks_per_thread": 2}
    prof = read_profile()
    same_shape = shape["impl"] == "ttable" and (shape["threads"], shape["blocks_per_thread"]) == prof["shape"]
    traffic = prof["traffic"].get(dom) if same_shape and n == NBLOCKS else None
    counters = dict(prof["ncu"][dom], source=prof["source"]) if same_shape and dom in prof["ncu"] else None
    kname = (f"tt_kernel<10,{dom},{shape['threads']},{shape['blocks_per_thread']}>" if shape["impl"] == "ttable"
             else f"bs_kernel<10,{dom}>")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "ncu": counters,
                "peak_source": f"derived: {sms} SMs x {SM_MAX_MHZ_NOMINAL:.0f} MHz x {blocks_per_sm_clock():.4f} blocks/SM-clock x 16 B",
                "enc_gbs": n * 16 / (enc_avg / 1e3) / 1e9, "dec_gbs": n * 16 / (dec_avg / 1e3) / 1e9,
                "enc_gbs_median": n * 16 / (statistics.median(enc_ms) / 1e3) / 1e9,
                "dec_gbs_median": n * 16 / (statistics.median(dec_ms) / 1e3) / 1e9,
                "enc_gbs_best": n * 16 / (min(enc_ms) / 1e3) / 1e9, "dec_gbs_best": n * 16 / (min(dec_ms) / 1e3) / 1e9,
                "hbm_term_gbs": hbm_peak_gbs() / 2,
                # the T-table design's own ceiling: 160 lookups (5 wavefronts) plus the block's
                # 16-byte load and store (1/8 wavefront each) through the L1/shared-memory path
                "lds_path_bound_gbs": lds_path_bound_gbs(sms, SM_MAX_MHZ_NOMINAL, ttable_wavefronts(10))}
    roofline["frac_of_lds_path_bound"] = achieved / roofline["lds_path_bound_gbs"]

    # ---- the same launches in place (output over input), outside the timed region ------------
    in_place = None
    extras = rank == 0 and world == 1  # single-GPU measurements, reported at N = 1 only
    if extras:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ip_enc, ip_dec = [], []
        for _ in range(10):
            ev[0].record(stream)
            st = lib.aes_crypt_blocks(ctypes.byref(ks), None, pp, pp, n, 0, impl, sptr)
            ev[1].record(stream)
            st |= lib.aes_crypt_blocks(ctypes.byref(ks), None, pp, pp, n, 1, impl, sptr)
            ev[2].record(stream)
            torch.cuda.synchronize()
            if st != 0:
                raise RuntimeError(aes.aes_last_error())
            ip_enc.append(ev[0].elapsed_time(ev[1]))
            ip_dec.append(ev[1].elapsed_time(ev[2]))
        if not torch.equal(pt, x):
            raise RuntimeError("in-place round trip failed")
        in_place = {"encrypt_gbs_median": n * 16 / (statistics.median(ip_enc) / 1e3) / 1e9,
                    "decrypt_gbs_median": n * 16 / (statistics.median(ip_dec) / 1e3) / 1e9,
                    "encrypt_gbs_best": n * 16 / (min(ip_enc) / 1e3) / 1e9,
                    "decrypt_gbs_best": n * 16 / (min(ip_dec) / 1e3) / 1e9, "repetitions": 10}

    bitsliced = None
    if extras and args.kernel != "bitslice" and not args.no_bitsliced:
        bitsliced = measure_bitsliced(aes, torch, dev, x, n, key, sms, local_rank)

    batched = None
    if not args.no_batched and extras:
        fixed = tuple(int(v) for v in args.batched_shape.split(",")) if args.batched_shape else None
        batched = measure_batched(aes, torch, dev, max(10, min(args.steps, 50)), roofline["enc_gbs"], fixed)

    followons = None
    if not args.no_followons and extras:
        followons = measure_followons(aes, torch, dev, x, n, key)
        followons["small_4096_blocks"] = measure_small_latency(aes, torch, dev)

    cbc = None
    if not args.no_cbc and extras:
        cbc = measure_cbc(aes, torch, dev)

    served = None
    if not args.no_served and extras:
        served = measure_served(aes, torch, dev, args.served_requests, roofline["enc_gbs"])

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
        cpu["openssl_context"] = openssl_ecb(w.key, w.data, cores, 3.0, gpu_ct[: 1 << 20])
        # the sensor column (10^7 records) on the same cores: a bounded sample of its records
        col = workloads.sensor_records(2, 10_000_000)
        for name, kb in (("aes128", col.key128), ("aes256", col.key256)):
            _, k = oracle_rate(orc, kb, col.records, cores, max(1.0, args.cpu_seconds / 4), 10_000_000)
            t = time.perf_counter()
            orc.encrypt_blocks(kb, col.records[: k * 16], threads=cores)
            cpu[f"sensor_{name}_encrypt_gbs"] = k * 16 / (time.perf_counter() - t) / 1e9
            cpu[f"sensor_{name}_records"] = k

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nblocks_per_rank": n, "key_bits": 128, "mode": "ECB (IV = 0)",
                       "kernel": args.kernel, "tuned": tuned, "l2": "inputs (1 GiB) larger than L2 (129 MB); no flush"},
            "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clk, "roofline": roofline,
            "cpu_baseline": cpu, "bitsliced": bitsliced, "batched": batched, "served": served, "cbc": cbc,
            "followons": followons, "in_place": in_place,
        }
        line["summary"] = summary_of(line, sms)  # last, so that a kept tail of the line holds it
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
