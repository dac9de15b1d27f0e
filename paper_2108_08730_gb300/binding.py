"""ctypes binding of libhx27 (include/hx27.h): argument marshalling only.

Device buffers are torch CUDA tensors (complex64 / complex128 / float32),
passed by data_ptr() with the current torch stream.  Every compute step runs
in the library's CUDA kernels; there is no Python or CPU fallback, and
``lib()`` raises if the shared library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhx27.so")

HX_OK = 0
STATUS = {0: "HX_OK", -1: "HX_ERR_ARG", -2: "HX_ERR_OOM", -3: "HX_ERR_NOT_CONVERGED",
          -4: "HX_ERR_NUMERIC", -5: "HX_ERR_TIMEOUT", -6: "HX_ERR_CUDA", -7: "HX_ERR_STATE",
          -8: "HX_ERR_CANCELLED"}

# every symbol include/hx27.h declares (checked by tests/test_abi.py)
EXPORTS = ("hx_build_weight_table", "hx_ctx_create", "hx_ctx_destroy", "hx_last_error",
           "hx_set_table", "hx_apply_operator", "hx_row_coefficients", "hx_assemble_csr",
           "hx_solve_default_opts", "hx_solve", "hx_profile", "hx_profile_read", "hx_measure_fp64_peak",
           "hx_assemble_csr_noalloc", "hx_kernel_config_info", "hx_set_kernel_config",
           "hx_autotune", "hx_stencil_sweep", "hx_server_create", "hx_server_submit",
           "hx_server_wait", "hx_server_get_stats", "hx_server_destroy", "hx_apply_batched",
           "hx_fit_joint_weights", "hx_set_table_ex", "hx_set_operator_form",
           "hx_set_medium", "hx_server_cancel", "hx_stencil_pitched")

NOALLOC_MAX_POINTS = 19683     # HX_NOALLOC_MAX_POINTS in include/hx27.h
APPLY_DIRECT = 0x100           # HX_APPLY_DIRECT in include/hx27.h

PROF_KINDS = {"apply32": 0, "smooth32": 1, "apply64": 2, "smooth64": 3}

SOLVE_MIXED, SOLVE_FP64 = 0, 1
SWEEP_RESIDUAL, SWEEP_JACOBI = 1, 2


class HxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class hx_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("f", C.c_double), ("npml", C.c_int * 6), ("v_ref", C.c_double),
                ("r_coef", C.c_double)]


class hx_source(C.Structure):
    _fields_ = [("ix", C.c_int), ("iy", C.c_int), ("iz", C.c_int), ("rhs", C.c_int),
                ("amp_re", C.c_double), ("amp_im", C.c_double)]


class hx_solve_opts(C.Structure):
    _fields_ = [("mode", C.c_int), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("max_outer", C.c_int), ("max_iter", C.c_int), ("shift_beta", C.c_double),
                ("mg_levels", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("coarse_sweeps", C.c_int), ("omega_jacobi", C.c_double),
                ("source_spread", C.c_int), ("initial_guess", C.c_int), ("check_every", C.c_int),
                ("coarse_galerkin", C.c_int), ("pml_cap", C.c_double), ("use_graphs", C.c_int),
                ("autotune", C.c_int), ("time_limit_s", C.c_double), ("cancel", C.c_void_p),
                ("nu_coarse", C.c_int), ("bicg_kappa", C.c_double), ("coarse_velocity", C.c_int)]


class hx_solve_report(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("inner_iters", C.c_int),
                ("mg_levels", C.c_int), ("rel_residual", C.c_double), ("setup_ms", C.c_double),
                ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hx_apply_item(C.Structure):
    _fields_ = [("grid", hx_grid), ("v_dev", C.c_void_p), ("x_dev", C.c_void_p), ("y_dev", C.c_void_p),
                ("nrhs", C.c_int)]


class hx_server_config(C.Structure):
    _fields_ = [("device", C.c_int), ("slots", C.c_int), ("mem_budget", C.c_double),
                ("table", C.POINTER(C.c_double)), ("n_g", C.c_int), ("d_inv_g", C.c_double),
                ("order", C.c_int), ("max_wait_s", C.c_double)]


class hx_request(C.Structure):
    _fields_ = [("model_id", C.c_uint64), ("v_host", C.c_void_p), ("grid", hx_grid),
                ("src", C.POINTER(hx_source)), ("nsrc", C.c_int), ("nrhs", C.c_int),
                ("wavefield_host", C.c_void_p), ("opts", C.POINTER(hx_solve_opts))]


class hx_request_result(C.Structure):
    _fields_ = [("status", C.c_int), ("report", hx_solve_report), ("queue_ms", C.c_double),
                ("run_ms", C.c_double), ("latency_ms", C.c_double), ("worker", C.c_int)]


class hx_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("point_rhs", C.c_double), ("busy_s", C.c_double), ("peak_committed", C.c_double),
                ("max_concurrent", C.c_int), ("cancelled", C.c_int64)]


_lib = None


def lib():
    """Load libhx27.so (built by ``paper_2108_08730_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2108_08730_gb300.build` (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, i, d, dp = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)
    L.hx_build_weight_table.argtypes = [dp, i, dp, i, d, d, d, dp, i, C.POINTER(C.c_int)]
    L.hx_fit_joint_weights.argtypes = [dp, i, dp, i, dp, i, dp]
    L.hx_ctx_create.argtypes = [C.POINTER(vp), i]
    L.hx_ctx_destroy.argtypes = [vp]
    L.hx_ctx_destroy.restype = None
    L.hx_last_error.argtypes = [vp]
    L.hx_last_error.restype = C.c_char_p
    L.hx_set_table.argtypes = [vp, dp, i, d]
    L.hx_set_table_ex.argtypes = [vp, dp, i, d, i]
    L.hx_set_operator_form.argtypes = [vp, i, i]
    L.hx_set_medium.argtypes = [vp, vp, vp]
    L.hx_apply_operator.argtypes = [vp, C.POINTER(hx_grid), vp, d, vp, vp, i, i, vp]
    L.hx_row_coefficients.argtypes = [vp, C.POINTER(hx_grid), vp, d, vp, vp]
    L.hx_assemble_csr.argtypes = [vp, C.POINTER(hx_grid), vp, d, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int32), dp, C.c_int64, C.POINTER(C.c_int64), vp]
    L.hx_solve_default_opts.argtypes = [C.POINTER(hx_solve_opts)]
    L.hx_solve_default_opts.restype = None
    L.hx_solve.argtypes = [vp, C.POINTER(hx_grid), vp, C.POINTER(hx_source), i, i, vp,
                           C.POINTER(hx_solve_opts), C.POINTER(hx_solve_report), vp]
    L.hx_assemble_csr_noalloc.argtypes = L.hx_assemble_csr.argtypes
    L.hx_stencil_sweep.argtypes = [vp, C.POINTER(hx_grid), vp, d, i, vp, vp, vp, i, i, d, vp]
    L.hx_measure_fp64_peak.argtypes = [vp, dp, vp]
    L.hx_stencil_pitched.argtypes = [vp, C.POINTER(hx_grid), vp, d, i, vp, vp, vp, i, C.c_int64, d, vp]
    L.hx_kernel_config_info.argtypes = [i, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.hx_set_kernel_config.argtypes = [vp, i]
    L.hx_autotune.argtypes = [vp, C.POINTER(hx_grid), vp, i, i, C.POINTER(C.c_int), dp, i, vp]
    L.hx_apply_batched.argtypes = [vp, C.POINTER(hx_apply_item), i, d, vp]
    L.hx_server_create.argtypes = [C.POINTER(vp), C.POINTER(hx_server_config)]
    L.hx_server_submit.argtypes = [vp, C.POINTER(hx_request), C.POINTER(C.c_int64)]
    L.hx_server_wait.argtypes = [vp, C.c_int64, d, C.POINTER(hx_request_result)]
    L.hx_server_get_stats.argtypes = [vp, C.POINTER(hx_server_stats), i]
    L.hx_server_cancel.argtypes = [vp, C.c_int64]
    L.hx_server_destroy.argtypes = [vp]
    L.hx_server_destroy.restype = None
    L.hx_profile.argtypes = [vp, i]
    L.hx_profile_read.argtypes = [vp, i, C.POINTER(C.c_int64), dp, dp]
    for name in EXPORTS:
        fn = getattr(L, name)
        if name not in ("hx_ctx_destroy", "hx_last_error", "hx_solve_default_opts", "hx_server_destroy"):
            fn.restype = C.c_int
    _lib = L
    return L


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def build_weight_table(theta_deg=(0, 10, 20, 30, 40, 45), phi_deg=(0, 10, 20, 30, 40, 45),
                       inv_g_max=0.4, d_inv_g=0.001, lam=1e-6):
    """hx_build_weight_table -> (inv_g nodes, table [n_g, 7]) as numpy FP64."""
    L = lib()
    th = np.ascontiguousarray(theta_deg, dtype=np.float64)
    ph = np.ascontiguousarray(phi_deg, dtype=np.float64)
    n_g = C.c_int(0)
    cap = 7 * (int(round(inv_g_max / d_inv_g)) + 1)
    out = np.zeros(cap, dtype=np.float64)
    st = L.hx_build_weight_table(_dptr(th), th.size, _dptr(ph), ph.size, inv_g_max, d_inv_g, lam,
                                 _dptr(out), cap, C.byref(n_g))
    if st != HX_OK:
        raise HxError(st, "hx_build_weight_table failed")
    T = out[:7 * n_g.value].reshape(n_g.value, 7)
    return np.arange(n_g.value) * d_inv_g, T


def fit_joint_weights(inv_g_list, theta_deg=(0, 10, 20, 30, 40, 45), phi_deg=(0, 10, 20, 30, 40, 45)):
    """hx_fit_joint_weights -> the 7 fixed weights of a non-adaptive stencil
    (G4: [1/4]; Gm: [1/4, 1/6, 1/8, 1/10])."""
    ig = np.ascontiguousarray(inv_g_list, dtype=np.float64)
    th = np.ascontiguousarray(theta_deg, dtype=np.float64)
    ph = np.ascontiguousarray(phi_deg, dtype=np.float64)
    w7 = np.zeros(7)
    st = lib().hx_fit_joint_weights(_dptr(ig), ig.size, _dptr(th), th.size, _dptr(ph), ph.size, _dptr(w7))
    if st != HX_OK:
        raise HxError(st, "hx_fit_joint_weights failed")
    return w7


def fixed_table(w7, n_g=401):
    """A weight table whose every node holds w7 (a non-adaptive stencil)."""
    return np.tile(np.asarray(w7, dtype=np.float64), (n_g, 1))


def kernel_configs():
    """[(rows per thread, RHS per CTA)] of the complex64 kernel configurations."""
    L = lib()
    n = L.hx_kernel_config_info(-1, None, None)
    out = []
    for c in range(n):
        a, b = C.c_int(0), C.c_int(0)
        L.hx_kernel_config_info(c, C.byref(a), C.byref(b))
        out.append((a.value, b.value))
    return out


def default_opts(**kw):
    """hx_solve_opts with the library defaults, overridden by keyword fields."""
    o = hx_solve_opts()
    lib().hx_solve_default_opts(C.byref(o))
    names = {k for k, _ in hx_solve_opts._fields_}
    for k, val in kw.items():
        if k not in names:
            raise KeyError(f"unknown solve option {k}")
        setattr(o, k, val)
    return o


def sources_of(workload, amp=1.0):
    """One unit source per RHS at the workload's source nodes."""
    return [(ix, iy, iz, r, amp) for r, (ix, iy, iz) in enumerate(workload.sources)]


def make_grid(shape, h, f, npml, v_ref, r_coef=1e-3):
    """hx_grid from (nz, ny, nx) and the rest."""
    nz, ny, nx = shape
    g = hx_grid()
    g.nx, g.ny, g.nz = int(nx), int(ny), int(nz)
    g.h, g.f = float(h), float(f)
    for k in range(6):
        g.npml[k] = int(npml[k])
    g.v_ref, g.r_coef = float(v_ref), float(r_coef)
    return g


def grid_of(workload):
    return make_grid(workload.shape, workload.h, workload.f, workload.npml, workload.v_ref,
                     workload.r_coef)


def _stream_ptr(stream):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns an hx_ctx on one CUDA device."""

    def __init__(self, device=0, table=None, d_inv_g=0.001):
        L = lib()
        h = C.c_void_p()
        st = L.hx_ctx_create(C.byref(h), int(device))
        if st != HX_OK:
            raise HxError(st, f"hx_ctx_create(device={device}) failed")
        self._h = h
        self.device = device
        if table is not None:
            self.set_table(table, d_inv_g)

    def close(self):
        if getattr(self, "_h", None):
            lib().hx_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != HX_OK:
            msg = lib().hx_last_error(self._h)
            raise HxError(st, f"{what}: {msg.decode() if msg else ''}")

    def set_table(self, table, d_inv_g=0.001, role="both"):
        """hx_set_table_ex with role "both", "operator" or "preconditioner"."""
        T = np.ascontiguousarray(table, dtype=np.float64)
        which = {"both": 0, "operator": 1, "preconditioner": 2}[role]
        self._check(lib().hx_set_table_ex(self._h, _dptr(T), T.shape[0], float(d_inv_g), which),
                    "hx_set_table_ex")

    def apply(self, grid, v, x, y, shift_beta=0.0, stream=None, direct=False):
        """y = A x; v float32 (nz,ny,nx) and x, y complex64/complex128
        (nrhs, nz, ny, nx) torch CUDA tensors.  direct=True selects the
        one-thread-per-row kernel (HX_APPLY_DIRECT)."""
        import torch
        prec = 32 if x.dtype == torch.complex64 else 64
        if direct:
            prec |= APPLY_DIRECT
        nrhs = x.shape[0] if x.dim() == 4 else 1
        self._check(lib().hx_apply_operator(self._h, C.byref(grid), C.c_void_p(v.data_ptr()),
                                            float(shift_beta), C.c_void_p(x.data_ptr()),
                                            C.c_void_p(y.data_ptr()), nrhs, prec, _stream_ptr(stream)),
                    "hx_apply_operator")

    def apply_batched(self, problems, shift_beta=0.0, stream=None):
        """hx_apply_batched: problems = [(grid, v, x, y)] with complex64 x, y
        (nrhs, nz, ny, nx) torch CUDA tensors; one persistent launch."""
        arr = (hx_apply_item * len(problems))()
        for k, (g, v, x, y) in enumerate(problems):
            arr[k] = hx_apply_item(g, C.c_void_p(v.data_ptr()), C.c_void_p(x.data_ptr()),
                                   C.c_void_p(y.data_ptr()), x.shape[0] if x.dim() == 4 else 1)
        self._check(lib().hx_apply_batched(self._h, arr, len(problems), float(shift_beta),
                                           _stream_ptr(stream)), "hx_apply_batched")

    def sweep(self, grid, v, kind, x, b, y, shift_beta=0.0, omega=0.6, stream=None):
        """hx_stencil_sweep: kind 'residual' (y = b - A x; b may be None) or
        'jacobi' (y = x + omega D^-1 (b - A x))."""
        import torch
        prec = 32 if x.dtype == torch.complex64 else 64
        nrhs = x.shape[0] if x.dim() == 4 else 1
        k = {"residual": SWEEP_RESIDUAL, "jacobi": SWEEP_JACOBI}[kind]
        bp = C.c_void_p(b.data_ptr()) if b is not None else C.c_void_p(0)
        self._check(lib().hx_stencil_sweep(self._h, C.byref(grid), C.c_void_p(v.data_ptr()),
                                           float(shift_beta), k, C.c_void_p(x.data_ptr()), bp,
                                           C.c_void_p(y.data_ptr()), nrhs, prec, float(omega),
                                           _stream_ptr(stream)), "hx_stencil_sweep")

    def row_coefficients(self, grid, v, coef, shift_beta=0.0, stream=None):
        self._check(lib().hx_row_coefficients(self._h, C.byref(grid), C.c_void_p(v.data_ptr()),
                                              float(shift_beta), C.c_void_p(coef.data_ptr()),
                                              _stream_ptr(stream)), "hx_row_coefficients")

    def solve(self, grid, v, sources, nrhs, out, stream=None, check=True, **opts):
        """hx_solve.  sources: [(ix, iy, iz, rhs, amp)] (amp complex), out:
        complex128 (nrhs, nz, ny, nx) torch CUDA tensor.  Keyword options are
        fields of hx_solve_opts.  Returns the report as a dict; raises HxError
        on failure unless check=False (then report['status'] carries it)."""
        o = default_opts(**opts)
        src = (hx_source * len(sources))()
        for k, (ix, iy, iz, rhs, amp) in enumerate(sources):
            a = complex(amp)
            src[k] = hx_source(int(ix), int(iy), int(iz), int(rhs), a.real, a.imag)
        rep = hx_solve_report()
        st = lib().hx_solve(self._h, C.byref(grid), C.c_void_p(v.data_ptr()), src, len(sources),
                            int(nrhs), C.c_void_p(out.data_ptr()), C.byref(o), C.byref(rep),
                            _stream_ptr(stream))
        if check:
            self._check(st, "hx_solve")
        return rep.as_dict()

    def set_operator_form(self, weights="GA", mass_form=2):
        """hx_set_operator_form: weights "GA" or "GAm", mass_form 2 or 1."""
        w = {"GA": 0, "GAm": 1}.get(weights, -1)
        self._check(lib().hx_set_operator_form(self._h, w, int(mass_form)), "hx_set_operator_form")

    def set_medium(self, buoyancy=None, inv_q=None):
        """hx_set_medium: float32 CUDA tensors (nz, ny, nx) of b = 1/rho and
        1/Q, or None.  The tensors are kept referenced until the next call."""
        self._medium = (buoyancy, inv_q)
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)
        self._check(lib().hx_set_medium(self._h, ptr(buoyancy), ptr(inv_q)), "hx_set_medium")

    def set_kernel_config(self, cfg):
        """Force a complex64 kernel configuration (-1: automatic)."""
        self._check(lib().hx_set_kernel_config(self._h, int(cfg)), "hx_set_kernel_config")

    def autotune(self, grid, v, nrhs, ncalls=3, stream=None):
        """hx_autotune -> (best configuration, [ms per launch by configuration])."""
        n = lib().hx_kernel_config_info(-1, None, None)
        best = C.c_int(-1)
        ms = (C.c_double * n)()
        self._check(lib().hx_autotune(self._h, C.byref(grid), C.c_void_p(v.data_ptr()), int(nrhs),
                                      int(ncalls), C.byref(best), ms, n, _stream_ptr(stream)),
                    "hx_autotune")
        return best.value, list(ms)

    def profile(self, enable=True):
        self._check(lib().hx_profile(self._h, 1 if enable else 0), "hx_profile")

    def profile_read(self):
        """{kind: (launches, total_ms, algo_bytes)} plus 'launches' (all kernels)."""
        out = {}
        n, ms, by = C.c_int64(0), C.c_double(0), C.c_double(0)
        for name, k in list(PROF_KINDS.items()) + [("all", -1)]:
            self._check(lib().hx_profile_read(self._h, k, C.byref(n), C.byref(ms), C.byref(by)),
                        "hx_profile_read")
            out[name] = (n.value, ms.value, by.value)
        return out

    def stencil_pitched(self, grid, v, kind, x, b, y, pitch, shift_beta=0.0, omega=0.6, stream=None):
        """hx_stencil_pitched on complex64 torch CUDA tensors (nrhs, nz, ny,
        pitch); kind "apply", "residual" or "jacobi"; b may be None for apply
        and residual."""
        k = {"apply": 0, "residual": 1, "jacobi": 2}[kind]
        nrhs = x.shape[0]
        bp = C.c_void_p(b.data_ptr()) if b is not None else None
        self._check(lib().hx_stencil_pitched(self._h, C.byref(grid), C.c_void_p(v.data_ptr()),
                                             float(shift_beta), k, C.c_void_p(x.data_ptr()), bp,
                                             C.c_void_p(y.data_ptr()), nrhs, int(pitch), float(omega),
                                             _stream_ptr(stream)), "hx_stencil_pitched")

    def fp64_peak(self, stream=None):
        """hx_measure_fp64_peak: measured FP64 FMA throughput in GFLOP/s."""
        g = C.c_double(0)
        self._check(lib().hx_measure_fp64_peak(self._h, C.byref(g), _stream_ptr(stream)),
                    "hx_measure_fp64_peak")
        return g.value

    def assemble_csr(self, grid, v, shift_beta=0.0, stream=None):
        """-> (rowptr int64, col int32, val complex128) numpy arrays."""
        N = grid.nx * grid.ny * grid.nz
        cap = 27 * N
        rowptr = np.zeros(N + 1, dtype=np.int64)
        col = np.zeros(cap, dtype=np.int32)
        val = np.zeros(2 * cap, dtype=np.float64)
        nnz = C.c_int64(0)
        self._check(lib().hx_assemble_csr(
            self._h, C.byref(grid), C.c_void_p(v.data_ptr()), float(shift_beta),
            rowptr.ctypes.data_as(C.POINTER(C.c_int64)), col.ctypes.data_as(C.POINTER(C.c_int32)),
            _dptr(val), cap, C.byref(nnz), _stream_ptr(stream)), "hx_assemble_csr")
        n = nnz.value
        return rowptr, col[:n].copy(), val[:2 * n].view(np.complex128).copy()

    def assemble_csr_noalloc(self, grid, v, shift_beta=0.0, stream=None):
        """hx_assemble_csr_noalloc: same result as assemble_csr without any
        device allocation by the library (grids of at most NOALLOC_MAX_POINTS
        points).  The numpy output arrays are host memory owned by Python."""
        N = grid.nx * grid.ny * grid.nz
        cap = 27 * N
        rowptr = np.zeros(N + 1, dtype=np.int64)
        col = np.zeros(cap, dtype=np.int32)
        val = np.zeros(2 * cap, dtype=np.float64)
        nnz = C.c_int64(0)
        self._check(lib().hx_assemble_csr_noalloc(
            self._h, C.byref(grid), C.c_void_p(v.data_ptr()), float(shift_beta),
            rowptr.ctypes.data_as(C.POINTER(C.c_int64)), col.ctypes.data_as(C.POINTER(C.c_int32)),
            _dptr(val), cap, C.byref(nnz), _stream_ptr(stream)), "hx_assemble_csr_noalloc")
        n = nnz.value
        return rowptr, col[:n].copy(), val[:2 * n].view(np.complex128).copy()


class Server:
    """hx_server: concurrent request serving of hx_solve on one device.

    Requests carry host arrays: the velocity (float32 (nz, ny, nx)) and the
    output wavefield (complex128 (nrhs, nz, ny, nx)); both are kept alive
    here until the request has been waited for."""

    def __init__(self, table, device=0, slots=2, mem_budget=0.0, d_inv_g=0.001, order="fifo",
                 max_wait_s=0.0):
        """order: "fifo" (first come, first served) or "smallest" (smallest
        request first; one waiting max_wait_s or longer goes first)."""
        self._T = np.ascontiguousarray(table, dtype=np.float64)
        o = {"fifo": 0, "smallest": 1}.get(order, -1)
        cfg = hx_server_config(int(device), int(slots), float(mem_budget), _dptr(self._T),
                               self._T.shape[0], float(d_inv_g), o, float(max_wait_s))
        h = C.c_void_p()
        st = lib().hx_server_create(C.byref(h), C.byref(cfg))
        if st != HX_OK:
            raise HxError(st, "hx_server_create failed")
        self._h = h
        self._keep = {}

    def submit(self, grid, v_host, sources, nrhs, out_host, model_id=0, **opts):
        """Queue one solve; returns its ticket.  sources as in Context.solve."""
        assert v_host.dtype == np.float32 and v_host.flags.c_contiguous
        assert out_host.dtype == np.complex128 and out_host.flags.c_contiguous
        src = (hx_source * len(sources))()
        for k, (ix, iy, iz, rhs, amp) in enumerate(sources):
            a = complex(amp)
            src[k] = hx_source(int(ix), int(iy), int(iz), int(rhs), a.real, a.imag)
        o = default_opts(**opts)
        req = hx_request(int(model_id), C.c_void_p(v_host.ctypes.data), grid, src, len(sources),
                         int(nrhs), C.c_void_p(out_host.ctypes.data), C.pointer(o))
        t = C.c_int64(-1)
        st = lib().hx_server_submit(self._h, C.byref(req), C.byref(t))
        if st != HX_OK:
            raise HxError(st, "hx_server_submit failed")
        self._keep[t.value] = (v_host, out_host)
        return t.value

    def wait(self, ticket, timeout=-1.0):
        """-> result dict (status, report, queue_ms, run_ms, latency_ms, worker)."""
        r = hx_request_result()
        st = lib().hx_server_wait(self._h, int(ticket), float(timeout), C.byref(r))
        if st == -5 and timeout >= 0:
            raise TimeoutError(f"request {ticket} still running")
        self._keep.pop(ticket, None)
        return {"status": r.status, "report": r.report.as_dict(), "queue_ms": r.queue_ms,
                "run_ms": r.run_ms, "latency_ms": r.latency_ms, "worker": r.worker}

    def cancel(self, ticket):
        """hx_server_cancel: the request completes with HX_ERR_CANCELLED (-8)."""
        st = lib().hx_server_cancel(self._h, int(ticket))
        if st != HX_OK:
            raise HxError(st, "hx_server_cancel failed")

    def stats(self, reset=False):
        s = hx_server_stats()
        st = lib().hx_server_get_stats(self._h, C.byref(s), 1 if reset else 0)
        if st != HX_OK:
            raise HxError(st, "hx_server_get_stats failed")
        return {k: getattr(s, k) for k, _ in hx_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().hx_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
