"""The seeded generators (inputs shared by the oracle's and the GPU path's
tests): determinism and the shapes/statistics their documentation states."""
import numpy as np

from paper_1411_2377_gb300 import synth


def test_splitmix64_reference_values():
    # splitmix64 with state 0: the first outputs of the published sequence
    z = synth._mix(np.array([0x9E3779B97F4A7C15, (2 * 0x9E3779B97F4A7C15) & ((1 << 64) - 1)],
                            dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_stencil_sizes():
    rp, ci, v = synth.stencil2d(64, seed=0)
    assert len(rp) - 1 == 4096 and rp[-1] == 20224
    rp, ci, v = synth.stencil2d(256, seed=0)
    assert rp[-1] == 326656
    rp, ci, v = synth.stencil3d(10, seed=2)
    assert len(rp) - 1 == 1000 and rp[-1] == 7 * 1000 - 6 * 100
    # rows are scaled by 10^(20 U): row maxima spread over ~20 decades
    mx = np.array([np.abs(v[rp[i]:rp[i + 1]]).max() for i in range(1000)])
    assert np.log10(mx.max() / mx.min()) > 15


def test_spmv_pattern_statistics():
    rp, ci = synth.random_csr_pattern(200_000, seed=1)
    n = len(rp) - 1
    lens = np.diff(rp)
    assert 14 < lens.mean() < 18 and lens.max() <= 256 and lens.min() >= 1
    rows = np.repeat(np.arange(n), lens)
    assert np.all(np.diff(ci.astype(np.int64)) [np.diff(rows) == 0] > 0)  # sorted, unique
    near = np.abs(ci - rows) <= 5000
    assert 0.88 < near.mean() < 0.93
    again = synth.random_csr_pattern(200_000, seed=1)
    assert np.array_equal(again[1], ci)


def test_random_values_encoding():
    v = synth.random_values(10000, 256, seed=4)
    heads = v[0].view(np.int64)
    zero = (heads >> 1) == synth.EXP_ZERO
    assert 0.005 < zero.mean() < 0.015
    e = heads[~zero] >> 1
    assert e.min() >= -39 and e.max() <= 41
    assert np.all(v[4][~zero] >> np.uint64(63) == 1)


def test_batch_systems_generator():
    d = synth.batch_systems(seed=3, count=256)
    assert len(d) == 256
    assert {x["p"] for x in d} == {128, 256}
    assert {x["kind"] for x in d} == {"2d", "3d"}
    assert all(1 <= x["nrhs"] <= 4 for x in d)
    ns = [x["m"] ** (2 if x["kind"] == "2d" else 3) for x in d]
    assert min(ns) >= 1000 and max(ns) <= 70000


def test_stencil_value_recipes():
    """The 5-point matrix: diagonal 4 + U(0, 0.1), neighbours -1 + 0.3 U(-1, 1)
    at the grid neighbours only; the 7-point convection-diffusion matrix:
    per row, diagonal 6 s and neighbours (-1 -/+ gamma) s with one scale s,
    gamma = Pe h / 2, the upwind side (-1 - gamma) towards lower indices."""
    m = 16
    rp, ci, v = synth.stencil2d(m, seed=0)
    rows = np.repeat(np.arange(m * m), np.diff(rp))
    diag = rows == ci
    assert np.all((v[diag] >= 4.0) & (v[diag] < 4.1))
    off = ~diag
    assert np.all((v[off] > -1.3) & (v[off] < -0.7))
    d = np.abs(ci[off].astype(np.int64) - rows[off])
    assert set(np.unique(d)) == {1, m}
    assert np.all((rows[off] // m == ci[off] // m) | (d == m))  # no wrap-around
    m, pe = 6, 50.0
    rp, ci, v = synth.stencil3d(m, seed=2, pe=pe)
    g = pe / (m + 1) / 2.0
    for i in range(m ** 3):
        s, e = rp[i], rp[i + 1]
        cols, vals = ci[s:e], v[s:e]
        scale = vals[cols == i][0] / 6.0
        assert 1.0 <= scale <= 1e20
        for c, a in zip(cols, vals):
            if c != i:
                want = (-1.0 - g) if c < i else (-1.0 + g)
                assert abs(a / scale - want) < 1e-12


def test_lotkin_pattern():
    """Section 3's workload: first row ones, a_ij = 1/(i+j-1) (1-based)
    below it, about s % of the entries dropped, the same draw for every
    precision (the pattern does not depend on p)."""
    n, s = 40, 30.0
    rp, ci, num, den = synth.lotkin_pattern(n, s, seed=7)
    assert np.all(num == 1.0)
    rows = np.repeat(np.arange(n), np.diff(rp))
    want = np.where(rows == 0, 1.0, rows + ci + 1.0)
    assert np.array_equal(den, want)
    kept = len(ci) / (n * n)
    assert 0.62 < kept < 0.78
    assert np.all(np.diff(ci.astype(np.int64))[np.diff(rows) == 0] > 0)
    full = synth.lotkin_pattern(n, 0.0, seed=7)
    assert full[0][-1] == n * n
    again = synth.lotkin_pattern(n, s, seed=7)
    assert all(np.array_equal(a, b) for a, b in zip(again, (rp, ci, num, den)))
