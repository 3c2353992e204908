"""Row-group plans of a skewed matrix: groups of 32 / (r * G) panels in which
one panel holds far more values than the others.  The heavy panel gets tiles
of its own (a segment tile, or pieces when it is longer than a tile) and the
group tile skips it, so the group's other panels stay in one tile.  Every
consumer of the row-group tiles is checked against the oracle: the SpMV
(1e-13 * sum_j |a_ij x_j|), the transposed product, the values gradient
(bit-exact) and the batched product."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2307_14774_gb300 as spc5
import synth
from gpuhelpers import assert_within_tol, convert, spmv, torch_cuda

pytestmark = pytest.mark.gpu

BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]


HEAVY, LONG = 211, 500


def _skewed(nrows=3000, ncols=60_000, seed=21):
    """Rows of up to 12 values near the diagonal; every 211th row holds about
    6,000 values (heavy: more than eight mean panels, even of eight rows),
    every 500th about 20,000 (longer than a tile)."""
    rng = np.random.default_rng(seed)
    rp, ci = [0], []
    for i in range(nrows):
        if i % LONG == 5:
            cols = np.flatnonzero(rng.random(ncols) < 1 / 3)
        elif i % HEAVY == 3:
            cols = np.flatnonzero(rng.random(ncols) < 0.1)
        else:
            k = int(rng.integers(0, 13))
            lo = min(max(0, 20 * i - 40), ncols - 100)
            cols = np.sort(lo + rng.choice(100, k, replace=False))
        ci.append(cols.astype(np.int32))
        rp.append(rp[-1] + len(cols))
    colidx = np.concatenate(ci)
    return synth.CSR(nrows, ncols, np.array(rp, np.int32), colidx, rng.normal(size=len(colidx)),
                     "skewed")


@pytest.fixture(scope="module")
def skewed():
    torch_cuda()
    return _skewed()


@pytest.mark.parametrize("log2g", [0, 2])
@pytest.mark.parametrize("r,c", BETAS)
def test_heavy_panels_leave_their_group(monkeypatch, skewed, r, c, log2g):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    monkeypatch.setenv("SPC5_LOG2G_GROUP", str(log2g))
    A = skewed
    M = convert(A, r, c)
    info = M.info()
    G = info["lanes_per_row"]
    groups = -(-info["npanels"] // (32 // (r * G)))
    heavy_rows = sum(1 for i in range(A.nrows) if i % LONG == 5 or i % HEAVY == 3)
    # one tile per group, plus the heavy panels' own tiles (pieces for the
    # longest): without the skip a fat group would give one tile per panel
    assert info["long_panels"] > 0
    assert info["ntiles"] <= groups + heavy_rows + info["pieces"]
    x = synth.vector_uniform(A.ncols, seed=2)
    y_ref, scale = oracle.csr_spmv(A, x)
    for body in ("0", "2", "5", "7"):
        monkeypatch.setenv("SPC5_BODY", body)
        Mb = convert(A, r, c)
        assert_within_tol(spmv(Mb, x), y_ref, scale)
    g = synth.vector_uniform(A.nrows, seed=3)
    ref_t, scale_t = oracle.csr_spmv_t(A, g)
    dx = torch.zeros(A.ncols, dtype=torch.float64, device="cuda")
    spc5.spc5_spmv_t(M, torch.from_numpy(g).cuda(), dx)
    torch.cuda.synchronize()
    assert_within_tol(dx.cpu().numpy(), ref_t, scale_t)
    dv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    spc5.spc5_values_grad(M, torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda(), dv)
    torch.cuda.synchronize()
    assert np.array_equal(dv.cpu().numpy(), oracle.values_grad(A, g, x))


@pytest.mark.parametrize("k", [1, 4])
def test_heavy_panels_batched(monkeypatch, skewed, k):
    torch = torch_cuda()
    monkeypatch.setenv("SPC5_KERNEL", "0")
    monkeypatch.setenv("SPC5_FLAT", "0")
    A = skewed
    Ms = [convert(A, r, c) for r, c in BETAS]
    X = synth.vector_uniform(A.ncols * k, seed=9).reshape(A.ncols, k)
    dX = [torch.from_numpy(X).cuda().contiguous() for _ in Ms]
    dY = [torch.full((A.nrows, k), float("nan"), dtype=torch.float64, device="cuda")
          for _ in Ms]
    spc5.spc5_spmv_batched(Ms, dX, dY, k)
    torch.cuda.synchronize()
    for Y in dY:
        Yh = Y.cpu().numpy()
        for j in range(k):
            y_ref, scale = oracle.csr_spmv(A, X[:, j])
            assert_within_tol(Yh[:, j], y_ref, scale)
