"""The seeded input recipes (paper_1506_08503_gb300/workloads.py), checked on the CPU against
what the benchmark and the parity tests claim about them: reproducible from the seed with the
keys drawn before the data, and the stated sizes and distributions (uniform bytes, the sensor
record layout, lognormal message lengths with a 4 KiB median, Poisson arrivals, the 50/50
direction mix and the half AES-128 / half AES-256 key pool)."""
import numpy as np
import pytest

from paper_1506_08503_gb300 import workloads


def test_plain_is_seeded_and_draws_the_key_first():
    a, b = workloads.plain(0, 4096), workloads.plain(0, 4096)
    assert (a.key == b.key).all() and (a.data == b.data).all()
    assert a.key.size == 16 and a.data.size == 4096 * 16 and a.data.dtype == np.uint8
    rng = np.random.default_rng(0)
    assert (a.key == rng.integers(0, 256, 16, dtype=np.uint8)).all()
    assert (workloads.plain(0, 64).data == a.data[:64 * 16]).all()  # a prefix of the same stream
    assert not (workloads.plain(1, 4096).data == a.data).all()
    # uniform bytes: every value appears, at close to 1/256 each
    counts = np.bincount(a.data, minlength=256)
    assert counts.min() > 0 and abs(counts.mean() - 256) < 1e-9 and counts.std() < 40


def test_sensor_records_layout_and_reading_distribution():
    n = 200_000
    col = workloads.sensor_records(2, n)
    rec = col.records.view("<i8").reshape(n, 2)
    assert col.key128.size == 16 and col.key256.size == 32
    assert (rec[:, 0] == 1_700_000_000_000_000_000 + np.arange(n, dtype=np.int64) * 1_000_000).all()
    r = rec[:, 1].astype(np.float64)
    assert abs(r.mean()) < 10 and 980 < r.std() < 1020 and (r == np.rint(r)).all()
    assert len(np.unique(rec[:, 1])) < n  # repeated readings: the equality scan has matches to find


def test_batched_messages_lengths():
    m = workloads.batched_messages(3)
    assert m.keys.shape == (4096, 16) and m.lengths.size == 4096
    assert (m.lengths % 16 == 0).all() and m.lengths.min() >= 16 and m.lengths.max() <= 16 << 20
    assert (m.offsets == np.concatenate([[0], np.cumsum(m.lengths)[:-1]])).all()
    assert m.data.size == m.lengths.sum()
    assert 3600 < np.median(m.lengths) < 4600  # lognormal, median 4 KiB (rounded up to blocks)
    assert 45e6 < m.lengths.sum() < 60e6       # about 52.6 MB
    logs = np.log(m.lengths[(m.lengths > 64) & (m.lengths < 1 << 20)])
    assert 1.3 < logs.std() < 1.6              # sigma 1.5 (clipping and rounding trim it a little)


@pytest.mark.parametrize("rate", [1000.0, 100000.0])
def test_served_requests_arrivals_and_mix(rate):
    n = 50_000
    w = workloads.served_requests(4, n, rate)
    assert len(w.pool_keys) == 1024
    assert all(k.size == 16 for k in w.pool_keys[:512]) and all(k.size == 32 for k in w.pool_keys[512:])
    gaps = np.diff(w.arrival_s)
    assert w.arrival_s[0] == 0 and (gaps >= 0).all()
    assert abs(gaps.mean() * rate - 1) < 0.02 and abs(gaps.std() * rate - 1) < 0.03  # exponential gaps
    assert abs(w.dirs.mean() - 0.5) < 0.01 and set(np.unique(w.dirs)) == {0, 1}
    assert w.key_idx.min() >= 0 and w.key_idx.max() < 1024 and abs((w.key_idx < 512).mean() - 0.5) < 0.01
    assert (w.lengths % 16 == 0).all() and w.lengths.min() >= 64 and w.lengths.max() <= 64 << 20
    # the same seed gives the same pool whatever the rate
    w2 = workloads.served_requests(4, 10, 7.0)
    assert all((a == b).all() for a, b in zip(w.pool_keys, w2.pool_keys))
