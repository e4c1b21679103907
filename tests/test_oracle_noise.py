"""Pins of the oracle's noise: Philox4x32-10, the uniform map, Box-Muller
normals and the Exp(1) thresholds of the first-passage test.

The random displacement R_i of Eq. 1 (Sec. II) has zero mean and covariance
2 D dt; each replica gets a unique random-number seed (Sec. II, RSF). Both are
realised with a counter-based Philox stream; these tests tie the oracle's
stream to an independent implementation of the published generator and to
the normal / exponential laws.

The independent implementation is the CUDA toolkit's host-side cuRAND
Philox4x32-10 generator (called through its C API, on the CPU). Its output
layout was established by comparison: the 64-bit seed is the key (low word
first), and output block b (four words) is the generator evaluated at the
counter (r, j, 0) with r, j = divmod(b, 65536), r a 64-bit pair of counter
words 0-1 and j counter word 2; the generator offset counts words. That
layout never reaches counter word 3, the chain id of the method's counter;
a second independent implementation, Triton's Philox4x32 (its own source,
run by its interpreter on the CPU, ``philox_triton_ref.py``), takes all four
words and pins the oracle there.
"""
import ctypes
import ctypes.util
import io
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
CURAND_LANES = 65536     # counter word 2 of consecutive output blocks


def _curand():
    names = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             ctypes.util.find_library("curand")]
    for n in names:
        if n:
            try:
                return ctypes.CDLL(n)
            except OSError:
                pass
    pytest.skip("cuRAND host library not found")


def _curand_blocks(seed, first_block, n_blocks):
    lib = _curand()
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                  ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out.reshape(n_blocks, 4)


def _counters_of(first_block, n_blocks):
    b = first_block + np.arange(n_blocks, dtype=np.uint64)
    r, j = b // CURAND_LANES, b % CURAND_LANES
    ctr = np.zeros((n_blocks, 4), dtype=np.uint32)
    ctr[:, 0] = (r & 0xFFFFFFFF).astype(np.uint32)
    ctr[:, 1] = (r >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = j.astype(np.uint32)
    return ctr


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 42])
def test_philox_matches_curand_over_two_counter_rounds(seed):
    # 2 x 65536 consecutive blocks: counter word 2 over its range, word 0 = 0, 1
    n = 2 * CURAND_LANES
    want = _curand_blocks(seed, 0, n)
    got = O.philox_many(_counters_of(0, n), [seed & 0xFFFFFFFF, seed >> 32])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("first_block", [CURAND_LANES * (1 << 32) + 5,             # counter word 1 = 1
                                         CURAND_LANES * 0x3F_FFFF_FFFF + 65500,    # words 0-1 and 2 near full
                                         123_456_789_012])
def test_philox_matches_curand_at_large_counters(first_block):
    seed = 0x9E3779B97F4A7C15
    want = _curand_blocks(seed, first_block, 64)
    got = O.philox_many(_counters_of(first_block, 64), [seed & 0xFFFFFFFF, seed >> 32])
    assert np.array_equal(got, want)


def _triton_blocks(ctr, seed):
    pytest.importorskip("triton")
    buf = io.BytesIO()
    np.save(buf, np.ascontiguousarray(ctr, dtype=np.uint32))
    script = os.path.join(os.path.dirname(os.path.abspath(__file__)), "philox_triton_ref.py")
    r = subprocess.run([sys.executable, script], input=buf.getvalue() + int(seed).to_bytes(8, "little"),
                       capture_output=True, timeout=600)
    assert r.returncode == 0, r.stderr.decode()[-2000:]
    return np.load(io.BytesIO(r.stdout))


def test_philox_matches_triton_on_all_four_counter_words():
    # random counters (every word, word 3 included) and the method's own
    # counters: (bead, slot | stream << 24, step, chain) with chain ids up to
    # 16383 in word 3, for two keys
    rng = np.random.default_rng(17)
    rand = rng.integers(0, 2**32, size=(1024, 4), dtype=np.uint64).astype(np.uint32)
    meth = np.zeros((1024, 4), dtype=np.uint32)
    meth[:, 0] = rng.integers(0, 512, size=1024)
    meth[:, 1] = rng.integers(0, 4097, size=1024) | (rng.integers(0, 2, size=1024) << 24)
    meth[:, 2] = rng.integers(0, 250_000, size=1024)
    meth[:, 3] = rng.integers(1, 16384, size=1024)
    ctr = np.concatenate([rand, meth])
    assert (ctr[:, 3] != 0).mean() > 0.99
    for seed in (0x0123456789ABCDEF, 5):
        want = _triton_blocks(ctr, seed)
        got = O.philox_many(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert np.array_equal(got, want)


def test_philox_batch_matches_single():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x12345678, 0x9abcdef0]
    many = O.philox_many(ctr, key)
    for j in range(0, 64, 7):
        assert np.array_equal(many[j], O.philox(ctr[j], key))


def test_uniform_open_interval_endpoints():
    assert O.uniform(0) == 2.0**-33
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0**-33
    assert O.uniform(0x80000000) == 0.5 + 2.0**-33
    # the 21-bit uniforms of the Box-Muller normals
    assert O.uniform21(0) == 2.0**-22
    assert O.uniform21(2**21 - 1) == 1.0 - 2.0**-22
    assert O.uniform21(2**20) == 0.5 + 2.0**-22


def _counters(n, slot=3, stream=0, step=11, chain=5):
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n) % 997
    ctr[:, 1] = slot | (stream << 24)
    ctr[:, 2] = step + np.arange(n) // 997
    ctr[:, 3] = chain
    return ctr


def test_normals_are_standard_normal():
    xi = O.normals3_many(42, _counters(120_000))
    n = xi.shape[0]
    for d in range(3):
        z = xi[:, d]
        assert abs(z.mean()) < 5.0 / np.sqrt(n)
        assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
        assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5.0 * np.sqrt(24.0 / n)
        assert stats.kstest(z, "norm").pvalue > 1e-4
    c = np.corrcoef(xi.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5.0 / np.sqrt(n))


def test_normals_depend_on_every_counter_word():
    base = O.normals3(7, 1, 2, 0, 3, 4)
    for args in [(8, 1, 2, 0, 3, 4), (7, 2, 2, 0, 3, 4), (7, 1, 3, 0, 3, 4),
                 (7, 1, 2, 1, 3, 4), (7, 1, 2, 0, 4, 4), (7, 1, 2, 0, 3, 5)]:
        assert not np.allclose(O.normals3(*args), base)
    assert np.array_equal(O.normals3(7, 1, 2, 0, 3, 4), base)


def test_replica_pairs_share_one_philox_output_as_three_box_muller_pairs():
    # Replicas 2j-1 and 2j draw the six normals of one Philox output (each
    # replica's own stream in law): their normals are the three Box-Muller
    # pairs (z0, z1), (z2, z3), (z4, z5) of slots (2j-1: z0 z1 z2, 2j: z3 z4
    # z5). A Box-Muller pair's squared radius is exponential with mean 2,
    # and all six are uncorrelated standard normals; a wrong half, a reused
    # angle or radius, or two replicas drawing the same half breaks one.
    n = 40_000
    for j in (1, 7):
        a = O.normals3_many(5, _counters(n, slot=2 * j - 1))
        b = O.normals3_many(5, _counters(n, slot=2 * j))
        z = np.concatenate([a, b], axis=1)                   # z0 .. z5
        r2 = np.array([z[:, 2 * k] ** 2 + z[:, 2 * k + 1] ** 2 for k in range(3)])
        for k in range(3):
            assert stats.kstest(r2[k], "expon", args=(0, 2.0)).pvalue > 1e-4, (j, k)
        cr = np.corrcoef(r2)                                 # independent radii
        assert np.all(np.abs(cr[np.triu_indices(3, 1)]) < 5.0 / np.sqrt(n))
        c = np.corrcoef(z.T)
        assert np.all(np.abs(c[np.triu_indices(6, 1)]) < 5.0 / np.sqrt(n))
        for d in range(6):
            assert stats.kstest(z[:, d], "norm").pvalue > 1e-4
        # 21-bit radial uniforms bound every normal by sqrt(-2 ln 2^-22)
        assert np.abs(z).max() <= np.sqrt(44.0 * np.log(2.0))
    # the parent (slot 0) has its own counter word (0), not a replica's
    p0 = O.normals3_many(5, _counters(1000, slot=0))
    p1 = O.normals3_many(5, _counters(1000, slot=1))
    assert not np.allclose(p0, p1)


def test_exp1_thresholds_are_unit_exponential():
    e = np.array([O.exp1(11, i, q, c) for c in range(40) for q in range(3) for i in range(100)])
    n = len(e)
    assert abs(e.mean() - 1.0) < 5.0 / np.sqrt(n)
    assert stats.kstest(e, "expon").pvalue > 1e-4
