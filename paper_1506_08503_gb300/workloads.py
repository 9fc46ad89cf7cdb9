"""Seeded synthetic inputs for the benchmark and the tests.

This module draws random bytes and sizes only; it holds none of the cipher's arithmetic, so
both the CUDA path and the CPU oracle can be fed from it.  Every generator takes its seed,
draws keys first and data after (a fixed order, so a workload is reproducible), and returns
numpy arrays.

The paper measures many 16-byte messages and 128 messages of varying length (Section IV,
Fig. 3) on no public dataset; these generators stand in for that workload:
  * plain(seed, nblocks)      one AES-128 key, nblocks uniform random blocks
  * sensor_records(seed, n)   16-byte records (int64 timestamp, int64 Gaussian reading)
  * batched_messages(seed)    4096 messages, lognormal lengths, one AES-128 key each
  * served_requests(seed)     Poisson arrivals of mixed encrypt/decrypt requests
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BLOCK = 16


def _bytes(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.integers(0, 256, size=n, dtype=np.uint8)


@dataclass
class Plain:
    key: np.ndarray   # (16,) uint8
    data: np.ndarray  # (nblocks*16,) uint8


def plain(seed: int, nblocks: int, key_bytes: int = 16) -> Plain:
    """One uniform random key, then nblocks uniform random blocks."""
    rng = np.random.default_rng(seed)
    key = _bytes(rng, key_bytes)
    return Plain(key=key, data=_bytes(rng, nblocks * BLOCK))


@dataclass
class SensorColumn:
    key128: np.ndarray
    key256: np.ndarray
    records: np.ndarray  # (n*16,) uint8: little-endian int64 timestamp, int64 reading


def sensor_records(seed: int, n: int, t0_ns: int = 1_700_000_000_000_000_000, cadence_ns: int = 1_000_000,
                   reading_std: float = 1000.0) -> SensorColumn:
    """An encrypted-database column: per record an int64 timestamp (t0 + i * cadence) and an
    int64 reading round(N(0, reading_std)), packed into one 16-byte block."""
    rng = np.random.default_rng(seed)
    key128 = _bytes(rng, 16)
    key256 = _bytes(rng, 32)
    readings = np.rint(rng.normal(0.0, reading_std, size=n)).astype("<i8")
    ts = (np.int64(t0_ns) + np.arange(n, dtype=np.int64) * np.int64(cadence_ns)).astype("<i8")
    rec = np.empty((n, 2), dtype="<i8")
    rec[:, 0] = ts
    rec[:, 1] = readings
    return SensorColumn(key128=key128, key256=key256, records=rec.view(np.uint8).reshape(-1))


@dataclass
class Messages:
    keys: np.ndarray     # (m, 16) uint8, one AES-128 key per message
    lengths: np.ndarray  # (m,) int64 bytes, multiples of 16
    offsets: np.ndarray  # (m,) int64 byte offsets into data (back to back)
    data: np.ndarray     # (sum(lengths),) uint8


def lognormal_lengths(rng: np.random.Generator, m: int, median: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    raw = rng.lognormal(mean=np.log(median), sigma=sigma, size=m)
    clipped = np.clip(raw, lo, hi)
    return (np.ceil(clipped / BLOCK) * BLOCK).astype(np.int64)


def batched_messages(seed: int, m: int = 4096, median: float = 4096.0, sigma: float = 1.5,
                     lo: int = 16, hi: int = 16 << 20, key_bytes: int = 16) -> Messages:
    """m messages with lognormal lengths (median 4 KiB, sigma 1.5, clipped to [16 B, 16 MiB],
    rounded up to whole blocks), each with its own random key, packed back to back."""
    rng = np.random.default_rng(seed)
    keys = _bytes(rng, m * key_bytes).reshape(m, key_bytes)
    lengths = lognormal_lengths(rng, m, median, sigma, lo, hi)
    offsets = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    data = _bytes(rng, int(lengths.sum()))
    return Messages(keys=keys, lengths=lengths, offsets=offsets, data=data)


@dataclass
class Requests:
    pool_keys: list          # list of uint8 arrays (16 or 32 bytes), the resident key pool
    arrival_s: np.ndarray    # (n,) float64 arrival times, seconds from start
    dirs: np.ndarray         # (n,) int32, 0 encrypt, 1 decrypt
    key_idx: np.ndarray      # (n,) int32 indices into pool_keys
    lengths: np.ndarray      # (n,) int64 bytes, whole blocks


def served_requests(seed: int, n: int, rate_hz: float, pool: int = 1024, median: float = 4096.0,
                    sigma: float = 1.5, lo: int = 64, hi: int = 64 << 20) -> Requests:
    """Poisson arrivals at rate_hz of a 50/50 encrypt/decrypt mix; sizes lognormal (median
    4 KiB, sigma 1.5) clipped to [64 B, 64 MiB] and rounded to whole blocks; keys drawn from a
    pool of `pool` keys, the first half AES-128 and the second half AES-256."""
    rng = np.random.default_rng(seed)
    pool_keys = [_bytes(rng, 16 if i < pool // 2 else 32) for i in range(pool)]
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    arrival = np.cumsum(gaps) - gaps[0]
    dirs = rng.integers(0, 2, size=n, dtype=np.int32)
    key_idx = rng.integers(0, pool, size=n, dtype=np.int32)
    lengths = lognormal_lengths(rng, n, median, sigma, lo, hi)
    return Requests(pool_keys=pool_keys, arrival_s=arrival, dirs=dirs, key_idx=key_idx, lengths=lengths)
