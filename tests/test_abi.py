"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/hx27.h declares, rejects bad arguments, and its host weight fit
(Section 2.2, banded Givens QR) matches the oracle's SVD least squares."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2108_08730_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(hx_\w+)\s*\(", src, re.M))
    return names


def test_header_declares_the_binding_exports():
    assert _declared() == set(B.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = B.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_weight_table_argument_errors():
    L = B.lib()
    th = np.zeros(3)
    out = np.zeros(10)
    n = C.c_int(0)
    dp = C.POINTER(C.c_double)
    st = L.hx_build_weight_table(th.ctypes.data_as(dp), 3, th.ctypes.data_as(dp), 3, 0.4, 0.001,
                                 1e-6, out.ctypes.data_as(dp), 10, C.byref(n))
    assert st == -1 and n.value == 401            # capacity too small, n_g reported
    st = L.hx_build_weight_table(th.ctypes.data_as(dp), 3, th.ctypes.data_as(dp), 3, 0.4, 0.001,
                                 0.0, out.ctypes.data_as(dp), 10, C.byref(n))
    assert st == -1                               # lambda must be > 0
    assert B.lib().hx_last_error(None) == b"no context"


@pytest.fixture(scope="module")
def tables():
    from oracle import weights as W
    return W.fit_table(), B.build_weight_table()


def test_host_fit_matches_oracle(tables):
    # Same regularised problem, different algorithms (oracle: dense SVD lstsq;
    # library: banded Givens QR).  The stacked system's condition number is
    # ~2.5e7 at lambda = 1e-6, so agreement to ~cond * eps (here 1e-8 on weights
    # of size ~1) is what FP64 allows.
    (nodes_o, To), (nodes_l, Tl) = tables
    assert Tl.shape == To.shape == (401, 7)
    assert np.allclose(nodes_o, nodes_l)
    assert np.max(np.abs(Tl - To)) < 1e-8


def test_host_fit_constraints_and_dispersion(tables):
    from oracle import weights as W
    _, (nodes, T) = tables
    assert np.max(np.abs(T[:, :3].sum(1) - 1)) < 1e-14
    assert np.max(np.abs(T[:, 3] + 6 * T[:, 4] + 12 * T[:, 5] + 8 * T[:, 6] - 1)) < 1e-14
    th, ph = W.angle_grid()
    for i in (25, 100, 250, 400):
        w_opt, _ = W.fit_per_g(nodes[i])
        e_opt = np.max(np.abs(W.phase_velocity(nodes[i], th, ph, W.expand_weights(w_opt)) - 1))
        e = np.max(np.abs(W.phase_velocity(nodes[i], th, ph, T[i]) - 1))
        assert e <= max(1.05 * e_opt, e_opt + 1e-6)


def test_ctx_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(B.HxError):
        B.Context(0)


@pytest.mark.parametrize("inv_g", [[0.25], [0.25, 1 / 6, 1 / 8, 0.1]])
def test_joint_fit_matches_oracle(inv_g):
    # the non-adaptive G4 / Gm weights (Eq. eq_cost): library normal-matrix
    # eigen-solve vs the oracle's SVD least squares (minimum norm for G4)
    from oracle import weights as W
    w7 = B.fit_joint_weights(inv_g)
    ref = W.expand_weights(W.fit_joint(inv_g).reshape(1, 5))[0]
    assert np.max(np.abs(w7 - ref)) < 1e-7
    assert abs(w7[0] + w7[1] + w7[2] - 1) < 1e-14
    assert abs(w7[3] + 6 * w7[4] + 12 * w7[5] + 8 * w7[6] - 1) < 1e-14


def test_context_setters_reject_a_null_context():
    # hx_set_operator_form / hx_set_medium / hx_set_kernel_config touch no GPU
    L = B.lib()
    assert L.hx_set_operator_form(None, 1, 1) == -1
    assert L.hx_set_medium(None, None, None) == -1
    assert L.hx_set_kernel_config(None, 0) == -1


def test_header_is_plain_c():
    # the boundary is a C ABI: the header must compile as C99 on its own,
    # and a C program must be able to link against the library's symbols
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "use.c")
        with open(src, "w") as f:
            f.write('#include "hx27.h"\n#include <stdio.h>\n'
                    "int main(void) { hx_solve_opts o; hx_solve_default_opts(&o);\n"
                    '  printf("%d %g\\n", o.max_iter, o.tol); return hx_last_error(0) == 0; }\n')
        out = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                              src, "-o", os.path.join(d, "use"), "-L", os.path.dirname(B.LIB_PATH), "-lhx27",
                              "-Wl,-rpath," + os.path.dirname(B.LIB_PATH)], capture_output=True, text=True)
        assert out.returncode == 0, out.stderr
        run = subprocess.run([os.path.join(d, "use")], capture_output=True, text=True, timeout=60)
        assert run.returncode == 0 and len(run.stdout.split()) == 2, (run.stdout, run.stderr)
