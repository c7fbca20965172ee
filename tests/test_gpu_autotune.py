"""Autotuned knobs on the GPU: every knob value gives the same C, bit for
bit (rows still accumulate over ascending k whichever accumulator or work
split they get), and the tuner returns a setting from its search space for a
product, a batch and a Galerkin chain."""
import numpy as np
import pytest

import oracle
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal, assert_values_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


TUNINGS = [dict(dense_min_flops=256), dict(dense_min_flops=32), dict(hash_shift=1),
           dict(hash_shift=2), dict(dense_chunk=2048), dict(dense_chunk=1024),
           dict(seg_log2=10), dict(seg_log2=22), dict(dense_min_flops=128, hash_shift=2,
                                                      dense_chunk=2048, seg_log2=12)]


@pytest.mark.parametrize("knobs", TUNINGS)
def test_every_knob_gives_the_same_product(sg, knobs):
    A = inputs.rmat(13, seed=41)
    dA = sg.to_device(A)
    base = sg.spgemm(dA, dA)
    t = sg.Tuning(**knobs)
    p = sg.plan(dA, dA, tuning=t)
    C = sg.spgemm(dA, dA, tuning=t, verify=True)
    assert bool((C.rowptr == base.rowptr).all()) and bool((C.col == base.col).all())
    assert bool((C.val == base.val).all())
    if "dense_min_flops" in knobs:
        assert p.info()["rows_dense"] > sg.plan(dA, dA).info()["rows_dense"]
    R = oracle.spgemm(A, A)
    assert_pattern_equal(C, R)
    assert_values_close(C, R, A, A)


@pytest.mark.parametrize("knobs", [dict(hash_shift=1), dict(dense_min_flops=64, hash_shift=2)])
def test_knobs_on_a_batch_and_a_device_sized_plan(sg, knobs):
    import torch
    As = [inputs.er_column_regular(n, d, 100 + n, value="u11_f32")
          for n, d in ((1024, 4), (2048, 16), (4096, 32))]
    dAs = [sg.to_device(A) for A in As]
    t = sg.Tuning(**knobs)
    Cs = sg.batch_spgemm(dAs, dAs, tuning=t, verify=True)
    ref = sg.batch_spgemm(dAs, dAs)
    for C, R in zip(Cs, ref):
        assert bool((C.col == R.col).all()) and bool((C.val == R.val).all())
    p = sg.device_plan(dAs[1:2], dAs[1:2], tuning=t)
    cap = 1 << 20
    rowptrC = torch.empty(p.R + 1, dtype=torch.int64, device="cuda")
    colC = torch.empty(cap, dtype=torch.int32, device="cuda")
    valC = torch.empty(cap, dtype=torch.float32, device="cuda")
    sg.execute(p, rowptrC, cap, colC, valC)
    sg.check(p)
    nnz = int(rowptrC[-1].item())
    assert bool((colC[:nnz] == ref[1].col).all()) and bool((valC[:nnz] == ref[1].val).all())


def test_tuner_on_a_product_and_a_batch(sg):
    from paper_1510_00844_gb300 import autotune
    A = inputs.rmat(12, seed=43)
    dA = sg.to_device(A)
    best, table = autotune.product(dA, dA, repeats=1)
    assert best in table and sg.Tuning() in table and len(table) >= 6
    for k, vals in autotune.SPACE.items():
        assert getattr(best, k) in tuple(vals) + (0,)
    assert table[best] <= table[sg.Tuning()]
    C = sg.spgemm(dA, dA, tuning=best)
    base = sg.spgemm(dA, dA)
    assert bool((C.val == base.val).all())
    As = [sg.to_device(inputs.er_column_regular(n, 8, n)) for n in (1024, 3000)]
    bb, bt = autotune.batch(As, As, repeats=1)
    assert bb in bt


def test_tuner_on_a_galerkin_chain(sg):
    import torch
    from paper_1510_00844_gb300 import amg, autotune
    N = 16
    A0 = sg.to_device(inputs.laplacian_7pt(N))
    Rs = [sg.to_device(inputs.aggregation_2x2x2(N >> l)) for l in range(2)]
    s = torch.cuda.Stream()
    best, table = autotune.galerkin(A0, Rs, s, repeats=2,
                                    space={"hash_shift": (0, 1, 2), "dense_min_flops": (1024, 32)})
    assert best in table and len(table) >= 4
    chain = amg.GalerkinChain(A0, Rs, s, tuning=best)
    chain.capture()
    chain.replay()
    torch.cuda.synchronize()
    chain.check()
    for l, C in enumerate(chain.results()):
        L = inputs.laplacian_7pt(N >> (l + 1))
        rp, col, val = C.to_host()
        assert np.array_equal(rp, L.rowptr) and np.array_equal(col, L.col)
        assert np.array_equal(val, L.val * 4.0 ** (l + 1))
