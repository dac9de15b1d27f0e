"""hx_assemble_csr_noalloc: the allocation-free variant of hx_assemble_csr.

Some callers cannot allocate device memory where they need the matrix (their
GPU memory belongs to another allocator, they must avoid cudaFree's device-wide
synchronisation, or their memory budget is fixed after start-up).  The variant
uses a fixed scratch array compiled into the library instead of a temporary
device buffer.  This file is collected last on purpose; it must pass alone in
a fresh process and after every other test.

Checks, with the oracle's weight table installed in the context so both sides
form the same operator:
  * two calls in a row on different grids, each equal to hx_assemble_csr
    (same structure, values within 1e-13 relative) and to the CPU oracle's
    CSR (oracle.operator.assemble_csr, same 1e-13);
  * grids at the limits: 2187 x 3 x 3 (the longest axis the per-axis scratch
    holds, every row of it filled) and 27^3, both exactly
    HX_NOALLOC_MAX_POINTS points, against the oracle;
  * a grid one plane above the limit is refused with a clear error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operator as O
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth

TOL = 1e-13


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


@pytest.fixture(scope="module")
def ctx(otable):
    c = B.Context(0)
    c.set_table(otable[1], 0.001)
    yield c
    c.close()


def _oracle_csr(otable, v, h, f, npml, vmax, beta):
    nodes, T = otable
    prof = O.profiles_for(v.shape, h, npml, vmax, 1e-3)
    return O.assemble_csr(v, h, f, prof, T, nodes, beta=beta)


def _check_against(rp, c, val, A):
    assert np.array_equal(rp, A.indptr) and np.array_equal(c, A.indices)
    assert np.max(np.abs(val - A.data)) <= TOL * np.max(np.abs(A.data))


def _case(k):
    if k == 0:
        shape, npml = (11, 10, 9), (2, 3, 1, 2, 3, 2)
    else:
        shape, npml = (20, 20, 20), (4, 4, 4, 4, 4, 4)
    return shape, npml, synth.random_velocity(shape, 50 + k, 1500.0, 3500.0)


def test_noalloc_matches_assemble_csr_and_oracle_twice(ctx, otable):
    for k, beta in ((0, 0.5), (1, 0.0)):            # two calls in a row, different grids
        shape, npml, v = _case(k)
        g = B.make_grid(shape, 25.0, 8.0, npml, 3500.0)
        vd = torch.from_numpy(v).cuda()
        rp0, c0, v0 = ctx.assemble_csr(g, vd, shift_beta=beta)
        rp1, c1, v1 = ctx.assemble_csr_noalloc(g, vd, shift_beta=beta)
        assert np.array_equal(rp0, rp1) and np.array_equal(c0, c1)
        assert np.max(np.abs(v1 - v0)) <= TOL * np.max(np.abs(v0))
        _check_against(rp1, c1, v1, _oracle_csr(otable, v, 25.0, 8.0, npml, 3500.0, beta))


@pytest.mark.parametrize("shape,npml", [((3, 3, 2187), (40, 37, 0, 0, 1, 1)),
                                        ((27, 27, 27), (5, 4, 3, 6, 2, 4))])
def test_noalloc_at_the_size_limit_matches_oracle(ctx, otable, shape, npml):
    assert int(np.prod(shape)) == B.NOALLOC_MAX_POINTS
    v = synth.random_velocity(shape, 77, 1500.0, 4000.0)
    g = B.make_grid(shape, 25.0, 6.0, npml, 4000.0)
    rp, c, val = ctx.assemble_csr_noalloc(g, torch.from_numpy(v).cuda(), shift_beta=0.25)
    _check_against(rp, c, val, _oracle_csr(otable, v, 25.0, 6.0, npml, 4000.0, 0.25))


def test_noalloc_rejects_grids_above_the_limit(ctx):
    g = B.make_grid((28, 27, 27), 25.0, 8.0, (2,) * 6, 3500.0)      # 20412 > 19683 points
    v = torch.full((28, 27, 27), 2000.0, device="cuda")
    with pytest.raises(B.HxError) as e:
        ctx.assemble_csr_noalloc(g, v)
    assert e.value.code == -1 and "HX_NOALLOC_MAX_POINTS" in str(e.value)
