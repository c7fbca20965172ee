"""Learned sizing on the GPU: the predictor's CUDA forward and backward
against the float64 reference, training that lowers the loss, and learned
products whose rows equal the two-phase path bit for bit -- with slots that
fit, with forced overflow (every row re-run), and for every value type."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1510_00844_gb300 import inputs
from tests.parity import assert_pattern_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available()
    from paper_1510_00844_gb300 import spgemm
    return spgemm


def test_forward_and_gradient_match_reference(sg):
    import torch
    rng = np.random.default_rng(3)
    N = 1000
    X = (rng.random((N, mlp.F)) * 12).astype(np.float32)
    t = (rng.random(N) * 10).astype(np.float32)
    p = (rng.normal(size=mlp.param_count()) * 0.2).astype(np.float32)
    dX, dt, dp = (torch.from_numpy(a).cuda() for a in (X, t, p))
    y = sg.sizer_forward(dX, dp).cpu().numpy()
    yr, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y, yr, rtol=1e-4, atol=1e-4)
    g, loss = sg.sizer_grad(dX, dt, dp)
    lr, gr = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss.item() - lr) <= 1e-4 * max(1, lr)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    big = np.abs(gr) > 1e-3 * np.abs(gr).max()
    np.testing.assert_allclose(g[big], gr[big], rtol=1e-3, atol=1e-5 * np.abs(gr).max())


def train_small(sg):
    pairs = [(inputs.rmat(s, seed=300 + s), None) for s in (9, 10, 11)]
    pairs += [(inputs.er_column_regular(2048, d, 400 + d), None) for d in (4, 8, 16)]
    dev = [(sg.to_device(A), sg.to_device(A)) for A, _ in pairs]
    X, T = sg.sizer_training_set(dev)
    params = sg.sizer_init(seed=1)
    trace = sg.sizer_train(X, T, params, steps=400, batch=1024, lr=3e-3, seed=2)
    return params, trace, X, T


def test_training_lowers_the_loss(sg):
    params, trace, X, T = train_small(sg)
    tr = trace.cpu().numpy()
    assert tr[-20:].mean() < 0.25 * tr[:20].mean()
    y = sg.sizer_forward(X, params)
    rmse = float(((y - T) ** 2).mean().sqrt())
    assert rmse < 1.0      # log2 units


@pytest.fixture(scope="module")
def trained(sg):
    return train_small(sg)[0]


@pytest.mark.parametrize("margin", [0.3, -4.0, 40.0])
def test_learned_product_equals_two_phase(sg, trained, margin):
    import torch
    A = inputs.rmat(12, seed=77)
    dA = sg.to_device(A)
    C, stats = sg.learned_multiply(dA, dA, trained, margin=margin)
    P = sg.spgemm(dA, dA)
    Cc = sg.compact(C)
    assert bool((Cc.rowptr == P.rowptr).all())
    assert bool((Cc.col == P.col).all()) and bool((Cc.val == P.val).all())
    if margin == -4.0:
        assert stats["overflow_rows"] > 0 and not stats["slots"]
    if margin == 40.0:
        assert stats["overflow_rows"] == 0 and stats["slots"]


@pytest.mark.parametrize("value", ["u11_f32", "int", "none"])
def test_learned_value_types(sg, trained, value):
    A = inputs.er_column_regular(4096, 12, 9, value=value)
    dA = sg.to_device(A)
    semiring = 1 if value == "none" else 0
    C, _ = sg.learned_multiply(dA, dA, trained, margin=0.1, semiring=semiring)
    P = sg.spgemm(dA, dA, semiring=semiring)
    Cc = sg.compact(C)
    assert bool((Cc.rowptr == P.rowptr).all()) and bool((Cc.col == P.col).all())
    if value != "none":
        assert bool((Cc.val == P.val).all())
    R = oracle.spgemm(A, A, semiring="or_and" if value == "none" else "plus_times")
    assert_pattern_equal(Cc, R)


@pytest.mark.parametrize("margin,value", [(40.0, "u01_f64"), (0.3, "u01_f64"), (-1.0, "u01_f64"),
                                          (0.3, "u11_f32"), (0.3, "int"), (0.3, "none")])
def test_learned_dense_rows_without_symbolic(sg, trained, margin, value):
    """Rows above the dense threshold take predicted slots too: their column
    segments (up to 8 per row at this scale) each fill a share of the slot and
    are packed together; a segment that outgrows its share sends the row to
    the exact re-run.  Rows equal the two-phase path bit for bit."""
    A = inputs.rmat(14, seed=91, value=value)
    dA = sg.to_device(A)
    semiring = 1 if value == "none" else 0
    p = sg.plan(dA, dA, semiring=semiring)
    inf = p.info()
    assert inf["rows_dense"] > 0 and inf["max_row_flops"] >= 1 << 18   # multi-segment rows
    C, stats = sg.learned_multiply(dA, dA, trained, margin=margin, semiring=semiring)
    P = sg.spgemm(dA, dA, semiring=semiring)
    Cc = sg.compact(C)
    assert bool((Cc.rowptr == P.rowptr).all()) and bool((Cc.col == P.col).all())
    if value != "none":
        assert bool((Cc.val == P.val).all())
    if margin == 40.0:
        assert stats["overflow_rows"] == 0 and stats["slots"]
    if margin == -1.0:
        assert stats["overflow_rows"] > 0


def test_learned_rerun_rows_go_to_spare_space(sg, trained):
    """With margin -40 every slot shrinks to its lower bound max_k |B(k,:)|:
    rows of A with one entry fit exactly, the ten rows with three entries
    overflow.  Their exact re-run output is small, so it lands in the spare
    space after the slots and C stays in slot form (no compaction)."""
    import numpy as np
    n = 4096
    perm = inputs.permutation(n, 5)
    rng = np.random.default_rng(6)
    rows = list(range(n))
    cols = list(perm)
    heavy = rng.choice(n, 10, replace=False)
    for r in heavy:
        for k in rng.choice(n, 2, replace=False):
            rows.append(int(r))
            cols.append(int(k))
    A = inputs.coo_to_csr(n, n, rows, cols, rng.random(len(rows)), index_dtype=np.int32)
    B = inputs.er_column_regular(n, 8, 7)
    dA, dB = sg.to_device(A), sg.to_device(B)
    C, stats = sg.learned_multiply(dA, dB, trained, margin=-40.0)
    assert 1 <= stats["overflow_rows"] <= 10 and stats["slots"]
    P = sg.spgemm(dA, dB)
    Cc = sg.compact(C)
    assert bool((Cc.rowptr == P.rowptr).all())
    assert bool((Cc.col == P.col).all()) and bool((Cc.val == P.val).all())


def test_rmat_scale20_panel_sampled_rows(sg):
    """The learned-sizing workload at full size: R-MAT scale 20 squaring on one
    row panel (1/16 of the rows, as the benchmark runs it) by the exact
    two-phase path and by learned sizing; the two agree bit for bit and a
    seeded sample of rows, including the panel's largest, matches the oracle
    row by row."""
    from tests.parity import rows_subset
    params = train_small(sg)[0]
    A = inputs.rmat(20)
    dA = sg.to_device(A)
    a, b = 0, A.nrows // 16
    view = sg.DeviceCSR(b - a, A.ncols, dA.rowptr[a:b], dA.col, dA.val, rowend=dA.rowptr[a + 1:b + 1])
    C = sg.spgemm(view, dA, verify=True)
    L, _ = sg.learned_multiply(view, dA, params, margin=0.35)
    Lc = sg.compact(L)
    assert bool((Lc.rowptr == C.rowptr).all()) and bool((Lc.col == C.col).all())
    assert bool((Lc.val == C.val).all())
    fl = oracle.row_flops(rows_subset(A, np.arange(a, b)), A)
    rng = np.random.default_rng(13)
    rows = np.unique(np.concatenate([np.argsort(-fl)[:4], rng.choice(b - a, 200, replace=False)]))
    R = oracle.spgemm(rows_subset(A, rows + a), A)
    rp, col, val = C.rowptr.cpu().numpy(), C.col.cpu().numpy(), C.val.cpu().numpy()
    for t, i in enumerate(rows):
        x, y = rp[i], rp[i + 1]
        u, v = R.rowptr[t], R.rowptr[t + 1]
        assert np.array_equal(col[x:y], R.col[u:v]) and np.array_equal(val[x:y], R.val[u:v])


def test_learned_with_a_broken_predictor_stays_exact(sg):
    """NaN parameters make every prediction NaN: capacities clamp to the
    exact lower bound max_k |B(k,:)| and rows that need more are re-run, so C
    still equals the two-phase product bit for bit (int64 indices here)."""
    import torch
    A = inputs.rmat(12, seed=97, index_dtype=np.int64)
    dA = sg.to_device(A)
    params = torch.full((sg.sizer_param_count(),), float("nan"), dtype=torch.float32,
                        device="cuda")
    C, stats = sg.learned_multiply(dA, dA, params, margin=0.3)
    P = sg.spgemm(dA, dA)
    Cc = sg.compact(C)
    assert stats["overflow_rows"] > 0
    assert bool((Cc.rowptr == P.rowptr).all()) and bool((Cc.col == P.col).all())
    assert bool((Cc.val == P.val).all())


def test_sizer_targets_match_row_counts(sg):
    """spgemm_sizer_targets gives log2(1 + nnz(C(i,:))) of the exact row counts
    (float32; the oracle's counts are exact integers)."""
    import torch
    A = inputs.rmat(10, seed=5)
    dA = sg.to_device(A)
    p = sg.plan(dA, dA)
    rp, _ = sg.symbolic(p)
    T = sg.sizer_targets(rp).cpu().numpy()
    R = oracle.spgemm(A, A)
    cnt = np.diff(np.asarray(R.rowptr)).astype(np.float64)
    np.testing.assert_allclose(T, np.log2(1.0 + cnt), rtol=2e-7, atol=2e-7)


def test_sizer_record_round_trip_gives_identical_learned_output(sg, trained):
    """A predictor saved to bytes and loaded back (as another process would)
    has the same parameters bit for bit and gives the same learned product."""
    import torch
    rec = sg.sizer_save(trained)
    assert rec[:7] == b"SGSIZER" and len(rec) == 8 + 24 + 4 * sg.sizer_param_count() + 8
    loaded = sg.sizer_load(rec)
    assert torch.equal(loaded.view(torch.int32), trained.view(torch.int32))
    A = inputs.rmat(11, seed=78)
    dA = sg.to_device(A)
    C1, s1 = sg.learned_multiply(dA, dA, trained, margin=0.3)
    C2, s2 = sg.learned_multiply(dA, dA, loaded, margin=0.3)
    a, b = sg.compact(C1), sg.compact(C2)
    assert s1["overflow_rows"] == s2["overflow_rows"]
    assert torch.equal(a.rowptr, b.rowptr) and torch.equal(a.col, b.col)
    assert torch.equal(a.val.view(torch.int64), b.val.view(torch.int64))
    bad = bytearray(rec)
    bad[40] ^= 1                                       # one flipped parameter bit
    with pytest.raises(sg.SpgemmError):
        sg.sizer_load(bytes(bad))
