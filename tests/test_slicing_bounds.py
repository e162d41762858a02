"""Arithmetic of the exact slicing the tensor-core factor relies on (Ozaki, Ogita, Oishi & Rump 2012).

The factor's TRSM and trailing updates split every double-float value h + l (|h + l| <= 2^e) into
six integer slices on the scale 2^(e - 8): h + l = 2^(e - 8) sum_s q_s 2^(-8 s) + rest.  Their
products are summed in FP32 on the tensor cores, level by level (l = s + t <= 5), and the sums must
be exact.  This file restates the splitting step in FP32 numpy (round to nearest even, a TwoSum
carrying the low word, as described) and checks the bounds the design rests on: |q_0| <= 256,
|q_s| <= 128 after it, every q_s exact in BF16, |rest| <= 2^(e - 49), and every level sum over a
64-wide panel at most 2^23.  No GPU involved.
"""
import numpy as np
import pytest

N_SLICES, BITS, PANEL = 6, 8, 64
f32 = np.float32


def slices(h, l, e):
    """Six slices of the pairs (h, l) (float32 arrays) on the scale 2^e (int array)."""
    sc = np.ldexp(np.ones_like(h), BITS - e).astype(f32)
    hh, ll = (h * sc).astype(f32), (l * sc).astype(f32)
    radix = f32(1 << BITS)
    q = []
    for _ in range(N_SLICES):
        qs = np.rint(hh).astype(f32)
        d = (hh - qs).astype(f32)
        s = (d + ll).astype(f32)
        bb = (s - d).astype(f32)
        err = ((d - (s - bb)) + (ll - bb)).astype(f32)
        q.append(qs)
        hh, ll = (s * radix).astype(f32), (err * radix).astype(f32)
    return np.stack(q)


def pairs(x):
    h = x.astype(f32)
    return h, (x - h.astype(np.float64)).astype(f32)


def bf16_exact(v):
    """True where the float32 value has at most 8 significant bits (exact in BF16)."""
    bits = v.astype(f32).view(np.uint32)
    return (bits & np.uint32(0xFFFF)) == 0


@pytest.fixture(scope="module")
def sample():
    rng = np.random.default_rng(20260)
    n = 200_000
    e = rng.integers(-6, 7, n)
    # magnitudes across 30 binades below the scale, both signs, and values at the scale itself
    x = rng.uniform(-1, 1, n) * np.ldexp(1.0, e) * np.exp2(-rng.uniform(0, 30, n))
    x[:1000] = np.ldexp(np.sign(rng.uniform(-1, 1, 1000)), e[:1000])
    return x, e


def test_slice_magnitudes_and_bf16(sample):
    x, e = sample
    h, l = pairs(x)
    q = slices(h, l, e)
    assert np.all(q == np.rint(q))
    assert np.abs(q[0]).max() <= 256
    assert np.abs(q[1:]).max() <= 128
    assert np.all(bf16_exact(q))


def test_slices_reconstruct_within_the_bound(sample):
    x, e = sample
    h, l = pairs(x)
    q = slices(h, l, e).astype(np.float64)
    recon = sum(q[s] * np.ldexp(1.0, -BITS * s) for s in range(N_SLICES)) * np.ldexp(1.0, e - BITS)
    value = h.astype(np.float64) + l.astype(np.float64)
    assert np.all(np.abs(value - recon) <= np.ldexp(1.0, e - 49))


def test_level_sums_are_exact_in_fp32():
    # worst case of a level l = s + t over a 64-wide panel: |q_0| <= 2^8, |q_s| <= 2^7 (s >= 1)
    for lev in range(N_SLICES):
        pairs_bound = sum((256 if s == 0 else 128) * (256 if lev - s == 0 else 128) for s in range(lev + 1))
        total = PANEL * pairs_bound
        assert total <= 2 ** 23 < 2 ** 24, (lev, total)
    # and on random slices: the FP32 sums of integer products equal the exact (int64) sums
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, (2, 512, PANEL))
    h, l = pairs(x)
    qa = slices(h[0].ravel(), l[0].ravel(), np.zeros(512 * PANEL, int)).reshape(N_SLICES, 512, PANEL)
    qb = slices(h[1].ravel(), l[1].ravel(), np.zeros(512 * PANEL, int)).reshape(N_SLICES, 512, PANEL)
    for lev in range(N_SLICES):
        exact = sum(qa[s].astype(np.int64) @ qb[lev - s].astype(np.int64).T for s in range(lev + 1))
        acc = np.zeros((512, 512), f32)
        for s in range(lev + 1):
            for k in range(PANEL):
                acc = (acc + np.outer(qa[s][:, k], qb[lev - s][:, k]).astype(f32)).astype(f32)
        assert np.array_equal(acc.astype(np.int64), exact)
