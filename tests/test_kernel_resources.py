"""Resource budget of the hot kernels, read from ptxas's own report
(nvcc -Xptxas -v: registers, stack frame, spill stores) when compiling for
sm_103a.  Needs nvcc, no GPU.

* st32_kernel with 1 or 2 RHS per CTA (the configurations of the 1- and
  2-RHS solves): no stack frame, no spills, at most 128 registers (two CTAs
  of 256 threads per SM);
* zm_frame_kernel (the PML rows of the tensor-copy kernel, all modes, with
  and without the shift): no stack frame, no spills, at most 168 registers
  (three CTAs of 128 threads per SM; its register window of four planes
  spilled at the 128-register cap of four CTAs);
* direct_stencil_k without a heterogeneous medium (every coarse multigrid
  level): no stack frame, no spills.  A stack frame here once came from an
  out-of-line call that took the row's 27 coefficients by address, and it
  slowed the coarse levels by about 10 %.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_08730_gb300", "csrc")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not available")


def _resources(src, tmp_path):
    out = subprocess.run(
        [_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c",
         os.path.join(CSRC, src), "-o", str(tmp_path / (src + ".o"))],
        capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res, cur = {}, None
    for line in out.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            cur = m.group(1)
            res[cur] = {}
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores", line)
        if m and cur:
            res[cur]["stack"], res[cur]["spill"] = int(m.group(1)), int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            res[cur]["regs"] = int(m.group(1))
    return res


_SOURCES = ("hx_stencil32.cu", "hx_galerkin.cu", "hx_zmarch_apply.cu", "hx_zmarch_residual.cu",
            "hx_zmarch_jacobi.cu")


@pytest.fixture(scope="module")
def resources(tmp_path_factory):
    """ptxas reports of the checked translation units, compiled in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    tmp = tmp_path_factory.mktemp("ptxas")
    _nvcc()
    with ThreadPoolExecutor(max_workers=len(_SOURCES)) as ex:
        return dict(zip(_SOURCES, ex.map(lambda src: _resources(src, tmp), _SOURCES)))


def test_complex64_stencil_budget(resources):
    res = resources["hx_stencil32.cu"]
    n = 0
    for name, r in res.items():
        m = re.search(r"st32_kernelILi(\d)ELi(\d)ELi(\d)E", name)
        if not m or int(m.group(3)) > 2:
            continue
        n += 1
        assert r.get("stack") == 0 and r.get("spill") == 0, (name, r)
        assert r.get("regs", 999) <= 128, (name, r)
    assert n == 6                                   # 3 modes x (1, 2 RHS per CTA)


def test_coarse_level_kernel_budget(resources):
    res = resources["hx_galerkin.cu"]
    n = 0
    for name, r in res.items():
        if re.search(r"direct_stencil_kI[fd]Li\dELb0E", name):
            n += 1
            assert r.get("stack") == 0 and r.get("spill") == 0, (name, r)
    assert n == 8                                   # 2 precisions x 4 modes


def test_frame_kernel_budget(resources):
    n = 0
    for src in ("hx_zmarch_apply.cu", "hx_zmarch_residual.cu", "hx_zmarch_jacobi.cu"):
        for name, r in resources[src].items():
            if "zm_frame_kernel" not in name:
                continue
            n += 1
            assert r.get("stack") == 0 and r.get("spill") == 0, (name, r)
            assert r.get("regs", 999) <= 168, (name, r)
    assert n == 6                                   # 3 modes x (shift, no shift)
