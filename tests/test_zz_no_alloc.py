"""hx_assemble_csr_noalloc: the allocation-free variant of hx_assemble_csr.

Some callers cannot allocate device memory where they need the matrix (their
GPU memory belongs to another allocator, they must avoid cudaFree's device-wide
synchronisation, or their memory budget is fixed after start-up).  The variant
uses a fixed scratch array compiled into the library instead of a temporary
device buffer.  This file is collected last on purpose; it must pass alone in
a fresh process and after every other test.

Check: two calls in a row, on two different grids, each compared with
hx_assemble_csr on the same inputs (same structure; values within the 1e-13
relative tolerance the coefficient tests use), plus the size limit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth


@pytest.fixture(scope="module")
def ctx():
    _, T = B.build_weight_table()
    c = B.Context(0, table=T)
    yield c
    c.close()


def _case(k):
    if k == 0:
        shape, npml = (11, 10, 9), (2, 3, 1, 2, 3, 2)
    else:
        shape, npml = (20, 20, 20), (4, 4, 4, 4, 4, 4)
    v = synth.random_velocity(shape, 50 + k, 1500.0, 3500.0)
    return B.make_grid(shape, 25.0, 8.0, npml, 3500.0), torch.from_numpy(v).cuda()


def test_noalloc_matches_assemble_csr_twice(ctx):
    for k, beta in ((0, 0.5), (1, 0.0)):            # two calls in a row, different grids
        g, v = _case(k)
        rp0, c0, v0 = ctx.assemble_csr(g, v, shift_beta=beta)
        rp1, c1, v1 = ctx.assemble_csr_noalloc(g, v, shift_beta=beta)
        assert np.array_equal(rp0, rp1) and np.array_equal(c0, c1)
        assert np.max(np.abs(v1 - v0)) <= 1e-13 * np.max(np.abs(v0))


def test_noalloc_rejects_grids_above_the_limit(ctx):
    g = B.make_grid((28, 27, 27), 25.0, 8.0, (2,) * 6, 3500.0)      # 20412 > 19683 points
    v = torch.full((28, 27, 27), 2000.0, device="cuda")
    with pytest.raises(B.HxError) as e:
        ctx.assemble_csr_noalloc(g, v)
    assert e.value.code == -1 and "HX_NOALLOC_MAX_POINTS" in str(e.value)
