"""Pins for the oracle's CDF tables and interleaved rANS coder (CPU only)."""
import math
import os

import numpy as np
import pytest

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_tables_invariants():
    freq, cum = oracle.build_tables()
    assert freq.shape == (64, 511) and cum.shape == (64, 512)
    assert (freq.sum(axis=1) == 65536).all()
    assert (freq >= 1).all()
    np.testing.assert_array_equal(freq, freq[:, ::-1])                  # symmetric in r
    np.testing.assert_array_equal(cum[:, 1:] - cum[:, :-1], freq)
    assert (cum[:, 0] == 0).all() and (cum[:, -1] == 65536).all()
    core = freq[:, 255:510]                                              # r = 0..254 (tail folded at 255)
    assert (np.diff(core.astype(np.int64), axis=1) <= 0).all()           # non-increasing in |r|


def test_table_smallest_scale_closed_form():
    """At s = 0.11 every r != 0 has p_r * (2^16 - 511) < 1, so f_r = 1 and f_0 = 2^16 - 510."""
    freq, _ = oracle.build_tables()
    p1 = 0.5 * math.erfc(0.5 / (0.11 * math.sqrt(2)))
    assert p1 * (65536 - 511) < 1
    assert freq[0, 255] == 65536 - 510
    assert (np.delete(freq[0], 255) == 1).all()


@pytest.mark.parametrize("k", [30, 40, 50, 63])
def test_table_entropy_matches_gaussian(k):
    """The table is a mixture (1 - e) p + e u of the discretised N(0, s^2) (entropy ~ 0.5 log2(2 pi e s^2)
    for s >= 2) and the e = 511/2^16 of mass that the "+1" floor spreads over all 511 symbols.  Mixture
    bounds: (1-e) H(p) <= H <= (1-e) H(p) + e log2(511) + h2(e).  Each f_r / 2^16 is also within the
    construction's rounding of the Gaussian pdf."""
    freq, _ = oracle.build_tables()
    s = oracle.scale(k)
    p = freq[k] / 65536.0
    H = -(p * np.log2(p)).sum()
    # integer-discretised Gaussian: entropy = 0.5 log2(2 pi e s^2) + log2(e)/(24 s^2) + o(1/s^2)
    # (Sheppard's correction for the midpoint rule)
    Hg = 0.5 * math.log2(2 * math.pi * math.e * s * s) + math.log2(math.e) / (24 * s * s)
    e = 511 / 65536
    h2 = -e * math.log2(e) - (1 - e) * math.log2(1 - e)
    assert (1 - e) * Hg - 0.002 <= H <= (1 - e) * Hg + e * math.log2(511) + h2 + 0.002
    if k == 63:
        assert abs(H - Hg) < 0.02
    # pointwise: against SciPy's Gaussian CDF (independent library routine), tails folded into +-255;
    # the floor moves < 1 count per symbol and the deficit (< 511 counts) lands on r = 0
    from scipy.stats import norm
    r = np.arange(-255, 256)
    pr = norm.cdf((r + 0.5) / s) - norm.cdf((r - 0.5) / s)
    pr[0] += norm.cdf(-254.5 / s)
    pr[-1] += norm.sf(254.5 / s)
    expect = 1 + pr * (65536 - 511)
    dev = freq[k].astype(np.float64) - expect
    assert (np.delete(dev, 255) <= 1e-6).all() and (np.delete(dev, 255) > -1 - 1e-6).all()
    assert 0 <= dev[255] < 511


def _golden(name):
    d = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or ":" not in line:
            continue
        k, v = line.split(":", 1)
        d[k.strip()] = v.split()
    return d


def test_rans_hand_derived_stream():
    g = _golden("rans_uniform_k1.txt")
    sym = np.array([int(v) for v in g["symbols"]], np.int16)
    want = bytes.fromhex("".join(g["section_hex"]))
    freq = np.full((1, 256), 256, np.uint32)
    cum = (np.arange(257, dtype=np.uint32) * 256)[None]
    tab = np.zeros(sym.size, np.uint8)
    got = oracle.rans_encode(sym, tab, 1, freq, cum, offset=0)
    assert got == want
    dec, used = oracle.rans_decode(got, tab, sym.size, 1, freq, cum, offset=0)
    np.testing.assert_array_equal(dec, sym)
    assert used == len(want)


@pytest.mark.parametrize("n,K", [(1000, 1), (1000, 7), (4096, 32), (33, 64), (0, 4)])
def test_rans_uniform_exact_bit_count(n, K):
    """Uniform 8-bit table: each lane of n_j symbols costs exactly 16*floor(n_j/2) + 32 bits."""
    rng = np.random.default_rng(n + K)
    sym = rng.integers(0, 256, n).astype(np.int16)
    freq = np.full((1, 256), 256, np.uint32)
    cum = (np.arange(257, dtype=np.uint32) * 256)[None]
    tab = np.zeros(n, np.uint8)
    bits = oracle.rans_encode(sym, tab, K, freq, cum, offset=0)
    counts = np.frombuffer(bits[:4 * K], np.uint32)
    nj = np.array([len(range(j, n, K)) for j in range(K)])
    np.testing.assert_array_equal(counts * 16, 16 * (nj // 2) + 32)
    dec, used = oracle.rans_decode(bits, tab, n, K, freq, cum, offset=0)
    np.testing.assert_array_equal(dec, sym)
    assert used == len(bits) and len(bits) % 4 == 0


@pytest.mark.parametrize("K", [1, 32, 1024])
def test_rans_gaussian_roundtrip_and_ideal(K):
    n = 60000
    r, b = synthetic.laplace_symbols(n, seed=K)
    thr = oracle.thresholds(32).astype(np.float64)
    idx = (thr[None, :] < np.log(b)[:, None]).sum(1).astype(np.uint8)
    freq, cum = oracle.build_tables()
    bits = oracle.rans_encode(r, idx, K, freq, cum)
    dec, used = oracle.rans_decode(bits, idx, n, K, freq, cum)
    np.testing.assert_array_equal(dec, r)
    assert used == len(bits)
    ideal = -np.log2(freq[idx, r.astype(np.int64) + 255] / 65536.0).sum()
    coded = 16 * np.frombuffer(bits[:4 * K], np.uint32).sum()
    # measured overhead of this 32-bit/16-bit-word coder stays well under 1 %, plus 32 flush bits/lane
    assert ideal - 32 * K <= coded <= ideal * 1.01 + 32 * K + 16


def test_rans_detects_corruption():
    n, K = 5000, 8
    r, b = synthetic.laplace_symbols(n, seed=3)
    idx = np.full(n, 30, np.uint8)
    bits = bytearray(oracle.rans_encode(r, idx, K))
    bad_count = bytearray(bits)
    bad_count[0] ^= 0x40                     # lane 0 claims a wrong number of words
    with pytest.raises(RuntimeError):
        oracle.rans_decode(bytes(bad_count), idx, n, K)
    with pytest.raises(RuntimeError):        # truncated stream
        oracle.rans_decode(bytes(bits[:len(bits) // 2]), idx, n, K)
    flipped = bytearray(bits)
    flipped[4 * K + 1] ^= 0x01               # initial state of lane 0 off by 256: final state check
    with pytest.raises(RuntimeError):
        oracle.rans_decode(bytes(flipped), idx, n, K)
