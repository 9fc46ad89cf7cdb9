"""Host-side logic of the library, checked on the CPU through the test hooks of
include/aesgb_testing.h (no GPU is touched): the batched launch's round-weighted warp
slicing, the request server's staging allocator, and the launch tuner's JSON cache.  Each is
checked against an independent model: numpy prefix sums of per-block work, a granule
occupancy map, and the json module."""
import ctypes
import json

import numpy as np
import pytest

_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_I8P = ctypes.POINTER(ctypes.c_int8)
_IP = ctypes.POINTER(ctypes.c_int)


@pytest.fixture(scope="module")
def hooks(aes):
    lib = aes.lib()
    lib.aes_testing_weighted_slices.restype = ctypes.c_int
    lib.aes_testing_weighted_slices.argtypes = [_U64P, _I8P, ctypes.c_size_t, ctypes.c_uint64, _U64P, _U32P]
    lib.aes_testing_arena.restype = ctypes.c_int
    lib.aes_testing_arena.argtypes = [ctypes.c_size_t, _I64P, ctypes.c_size_t, _I64P]
    lib.aes_testing_tune_cache_store.restype = ctypes.c_int
    lib.aes_testing_tune_cache_store.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_double]
    lib.aes_testing_cols_shape.restype = ctypes.c_int
    lib.aes_testing_cols_shape.argtypes = [ctypes.c_uint64, ctypes.c_int] + [ctypes.POINTER(ctypes.c_uint)] * 4
    lib.aes_testing_tune_cache_lookup.restype = ctypes.c_int
    lib.aes_testing_tune_cache_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, _IP, _IP, _IP]
    return lib


def _p(a, t):
    return a.ctypes.data_as(t)


def slices(hooks, nblocks, rounds, nw):
    nb = np.ascontiguousarray(nblocks, dtype=np.uint64)
    rd = np.ascontiguousarray(rounds, dtype=np.int8)
    gb = np.zeros(nw + 1, dtype=np.uint64)
    msg = np.zeros(nw, dtype=np.uint32)
    rc = hooks.aes_testing_weighted_slices(_p(nb, _U64P), _p(rd, _I8P), nb.size, nw, _p(gb, _U64P), _p(msg, _U32P))
    return rc, gb.astype(np.int64), msg.astype(np.int64)


@pytest.mark.parametrize("seed", range(12))
def test_weighted_slices_are_balanced_and_consistent(hooks, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    nblocks = np.maximum(1, rng.lognormal(5, 1.5, n)).astype(np.int64)
    rounds = rng.choice([10, 12, 14], n)
    nw = int(rng.integers(1, 2500))
    rc, gb, msg = slices(hooks, nblocks, rounds, nw)
    assert rc == 0
    start = np.concatenate([[0], np.cumsum(nblocks)])
    total = int(start[-1])
    assert gb[0] == 0 and gb[-1] == total and (np.diff(gb) >= 0).all()
    inside = gb[:-1] < total
    assert ((start[msg] <= gb[:-1]) & (gb[:-1] < start[msg + 1]))[inside].all()
    # work of every slice from an independent per-block prefix sum
    work = np.concatenate([[0], np.cumsum(np.repeat(rounds, nblocks))])
    per_slice = work[gb[1:]] - work[gb[:-1]]
    ideal = work[-1] / nw
    assert per_slice.sum() == work[-1]
    assert np.abs(per_slice - ideal).max() <= 14 + 1


def test_weighted_slices_equal_rounds_match_equal_block_cuts(hooks):
    # with one round count, equal work is equal blocks: warp w starts at floor(total * w / nw)
    nblocks = np.array([7, 1000, 3, 50_000, 1], dtype=np.int64)
    rc, gb, _ = slices(hooks, nblocks, np.full(5, 10), 333)
    total = int(nblocks.sum())
    want = np.array([total * w // 333 for w in range(334)])
    assert rc == 0 and (gb == want).all()


def test_weighted_slices_reject_bad_input(hooks):
    assert slices(hooks, [5, 0, 3], [10, 10, 10], 4)[0] == -1  # an empty message
    assert slices(hooks, [5, 3], [10, 11], 4)[0] == -1  # not an AES round count


def arena(hooks, size, ops):
    o = np.ascontiguousarray(ops, dtype=np.int64)
    res = np.zeros(o.size, dtype=np.int64)
    rc = hooks.aes_testing_arena(size, _p(o, _I64P), o.size, _p(res, _I64P))
    return rc, res


@pytest.mark.parametrize("seed", range(8))
def test_arena_first_fit_with_coalescing(hooks, seed):
    rng = np.random.default_rng(100 + seed)
    size = 256 * int(rng.integers(64, 512))
    ops, live = [], []
    for i in range(400):
        if live and rng.random() < 0.45:
            j = live.pop(int(rng.integers(0, len(live))))
            ops.append(-(j + 1))
        else:
            ops.append(int(rng.integers(1, size // 6)))
            live.append(i)
    rc, res = arena(hooks, size, ops)
    assert rc == 0
    # replay on a granule occupancy map
    granules = size // 256
    used = np.zeros(granules, dtype=bool)
    held = {}
    for i, op in enumerate(ops):
        if op > 0:
            g = -(-op // 256)
            runs = np.flatnonzero(np.convolve(~used, np.ones(g, dtype=int), "valid") == g) if g <= granules else []
            # first fit over maximal free runs: the lowest start of a free run that holds g granules
            first = None
            k = 0
            while k < granules:
                if used[k]:
                    k += 1
                    continue
                e = k
                while e < granules and not used[e]:
                    e += 1
                if e - k >= g:
                    first = k
                    break
                k = e
            if first is None:
                assert res[i] == -1 and len(runs) == 0
            else:
                assert res[i] == 256 * first
                assert not used[first:first + g].any()
                used[first:first + g] = True
                held[i] = (first, g)
        else:
            j = -op - 1
            if j in held:
                s, g = held.pop(j)
                used[s:s + g] = False


def test_arena_rejects_bad_operations(hooks):
    assert arena(hooks, 4096, [256, -2])[0] == -1  # frees an operation that comes later
    assert arena(hooks, 4096, [256, -1, -1])[0] == -1  # double free
    assert arena(hooks, 4096, [0])[0] == -1


def test_tune_cache_store_and_lookup(hooks, tmp_path):
    path = str(tmp_path / "tune.json").encode()
    i, t, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert hooks.aes_testing_tune_cache_lookup(path, b"dev|enc|nr10|log2n26", ctypes.byref(i), ctypes.byref(t),
                                               ctypes.byref(u)) == 0
    assert hooks.aes_testing_tune_cache_store(path, b"dev|enc|nr10|log2n26", 1, 768, 2, 1160.5) == 0
    assert hooks.aes_testing_tune_cache_store(path, b"dev|dec|nr14|log2n20", 2, 128, 32, 80.0) == 0
    assert hooks.aes_testing_tune_cache_store(path, b"dev|dec|nr12|log2n20", 1, 500, 2, 80.0) == 0  # not compiled
    entries = json.loads(open(path, "rb").read())
    assert set(entries) == {"dev|enc|nr10|log2n26", "dev|dec|nr14|log2n20", "dev|dec|nr12|log2n20"}
    assert entries["dev|enc|nr10|log2n26"] == {"impl": 1, "threads": 768, "unroll": 2, "us": 1160.5}
    assert hooks.aes_testing_tune_cache_lookup(path, b"dev|enc|nr10|log2n26", ctypes.byref(i), ctypes.byref(t),
                                               ctypes.byref(u)) == 1
    assert (i.value, t.value, u.value) == (1, 768, 2)
    assert hooks.aes_testing_tune_cache_lookup(path, b"dev|dec|nr14|log2n20", ctypes.byref(i), ctypes.byref(t),
                                               ctypes.byref(u)) == 1
    assert (i.value, t.value, u.value) == (2, 128, 32)
    # an entry that names no compiled candidate is ignored, so the tuner times instead
    assert hooks.aes_testing_tune_cache_lookup(path, b"dev|dec|nr12|log2n20", ctypes.byref(i), ctypes.byref(t),
                                               ctypes.byref(u)) == 0


def cols_shape(hooks, chains, sms):
    v = [ctypes.c_uint() for _ in range(4)]
    rc = hooks.aes_testing_cols_shape(chains, sms, *[ctypes.byref(x) for x in v])
    assert rc == 0
    return tuple(x.value for x in v)  # threads, chain warps per CTA, grid, chains per warp


@pytest.mark.parametrize("sms", [1, 7, 152])
def test_cbc_cols_shape_covers_every_chain_in_one_pass(hooks, sms):
    """The four-lanes-per-chain CBC launch for 1 .. 64 x sms chains: at most one CTA per SM, at
    least 128 threads (the table fill), chain warps that fit the CTA, 1-8 chains per warp, one
    chain per warp while there are at most 4 per SM, and enough chain slots for every chain at
    once (the chains run side by side, none waits for another to finish)."""
    for chains in list(range(1, 4 * sms + 2)) + [32 * sms, 32 * sms + 1, 64 * sms - 1, 64 * sms]:
        threads, wpc, grid, cpw = cols_shape(hooks, chains, sms)
        assert 1 <= grid <= sms and 1 <= wpc <= 8 and 1 <= cpw <= 8, chains
        assert threads == max(128, 32 * wpc), chains
        assert grid * wpc * cpw >= chains, chains
        if chains <= 4 * sms:
            assert cpw == 1, chains
    assert hooks.aes_testing_cols_shape(0, sms, *[ctypes.byref(ctypes.c_uint()) for _ in range(4)]) == -1

