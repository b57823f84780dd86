"""Launch configurations and the autotuner: every configuration of a
matrix's products gives the oracle's result bit for bit, the tuner keeps one
of them, and the on-disk cache reproduces it without timing again."""
import json

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitwise, need_gpu, rand_planes, random_csr, recs

pytestmark = pytest.mark.gpu
MODES = (("ordered", oracle.ORDERED), ("exact", oracle.EXACT))


@pytest.mark.parametrize("p", (128, 256, 512, 1024))
def test_every_configuration_matches_the_oracle(p):
    mpk = need_gpu()
    n = 2113 if p <= 256 else 803
    rowptr, colidx = random_csr(n, seed=p + 1, mean_len=9, max_len=120, empty_every=13)
    V = rand_planes(len(colidx), p, 31, zero_frac=0.05, emin=-30, emax=30)
    X = rand_planes(n, p, 32, zero_frac=0.05, emin=-30, emax=30)
    A = mpk.CSR(rowptr, colidx, V, p, transpose=True)
    x = mpk.Vec.from_planes(X, p)
    for name, m in MODES:
        want, st = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        want_t, _ = oracle.spmv_t(p, m, rowptr, colidx, recs(V), recs(X))
        stagings = (0, 1, -1) if name == "ordered" else (-1,)
        for tpb in (32, 64, 128, 256):
            for s in stagings:
                A.set_config(name, tpb, s)
                got = A.get_config(name)
                assert got["threads_per_block"] == tpb
                what = f"{name} p={p} tpb={tpb} staging={s}"
                assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, what)
                assert_bitwise(mpk.spmv_t(A, x, mode=name).planes(), want_t, "T " + what)


def test_bad_configuration_is_rejected():
    mpk = need_gpu()
    rowptr, colidx = random_csr(64, seed=2)
    A = mpk.CSR(rowptr, colidx, np.ones(len(colidx)), 128)
    for args in (("ordered", 96, -1), ("ordered", 128, 2), ("exact", 512, -1)):
        with pytest.raises(mpk.MPError):
            A.set_config(*args)
    assert A.get_config("ordered")["threads_per_block"] == 128


@pytest.mark.parametrize("p", (128, 1024))
def test_tuner_and_cache(p, tmp_path):
    mpk = need_gpu()
    from paper_1411_2377_gb300 import tune

    n = 20000
    rowptr, colidx = random_csr(n, seed=7, mean_len=8, max_len=64, band=300)
    V = rand_planes(len(colidx), p, 41, emin=-10, emax=10)
    X = rand_planes(n, p, 42, emin=-10, emax=10)
    A = mpk.CSR(rowptr, colidx, V, p)
    x = mpk.Vec.from_planes(X, p)
    cache = str(tmp_path / "tune.json")
    first = tune.autotune(A, reps=2, cache=cache)
    for name, m in MODES:
        r = first[name]
        assert not r["cached"] and r["ms"] > 0
        assert r["threads_per_block"] in (32, 64, 128, 256)
        assert A.get_config(name)["threads_per_block"] == r["threads_per_block"]
        if name == "ordered":
            assert r["staging"] in ((0, 1) if p <= 512 else (0,))
        want, _ = oracle.spmv(p, m, rowptr, colidx, recs(V), recs(X))
        assert_bitwise(mpk.spmv(A, x, mode=name).planes(), want, f"tuned {name} p={p}")
    assert len(json.load(open(cache))) == 2
    B = mpk.CSR(rowptr, colidx, V, p)
    again = tune.autotune(B, reps=2, cache=cache)
    for name, _ in MODES:
        assert again[name]["cached"]
        assert B.get_config(name) == A.get_config(name)
