"""Thin ctypes binding of the C ABI in include/condipm.h.

Argument marshalling only: every computation runs in the CUDA kernels of
libcondipm.so.  Device vectors are passed as torch CUDA tensors (float64,
contiguous); PyTorch only supplies device memory and streams.  The binding
raises if the library is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcondipm.so")

OPF_OK = 0
OPF_ERR_INVALID_ARG = -1
OPF_ERR_CUDA = -2
OPF_ERR_NOT_PD = -3
OPF_ERR_SINGULAR = -4
OPF_ERR_PF_FAILED = -5
OPF_ERR_TIMEOUT = -6
OPF_ERR_NO_CONVERGENCE = -8
OPF_ERR_INFEASIBLE = -9
OPF_ROUTE_ADJOINT = 0
OPF_ROUTE_EXPLICIT = 1
OPF_ROUTE_AUTO = 2
OPF_VEC_F, OPF_VEC_G, OPF_VEC_H, OPF_VEC_GRADF = 0, 1, 2, 3
OPF_MAT_G, OPF_MAT_A, OPF_MAT_W, OPF_MAT_K = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class opf_network(C.Structure):
    _fields_ = [("nb", C.c_int), ("nl", C.c_int), ("ng", C.c_int), ("slack", C.c_int),
                ("Pd", _dp), ("Qd", _dp), ("Vmin", _dp), ("Vmax", _dp),
                ("lf", _ip), ("lt", _ip), ("r", _dp), ("x", _dp), ("b", _dp), ("rate", _dp),
                ("gbus", _ip), ("Pmin", _dp), ("Pmax", _dp), ("Qmin", _dp), ("Qmax", _dp),
                ("c2", _dp), ("c1", _dp)]


class opf_options(C.Structure):
    _fields_ = [("route", C.c_int), ("rhs_block", C.c_int), ("spin_limit", C.c_longlong),
                ("chol_form", C.c_int), ("rhs1_kernel", C.c_int), ("rhs_width", C.c_int),
                ("dense_forward", C.c_int)]


class opf_ipm_options(C.Structure):
    _fields_ = [("variant", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("mu0", C.c_double),
                ("pf_tol", C.c_double), ("verbose", C.c_int), ("line_search", C.c_int),
                ("restoration", C.c_int), ("start_with_resto", C.c_int), ("linear_solver", C.c_int)]


class opf_ipm_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("obj", C.c_double), ("err", C.c_double),
                ("mu", C.c_double), ("n_factor", C.c_int), ("ms_total", C.c_double), ("ms_eval", C.c_double),
                ("ms_condense", C.c_double), ("ms_factor", C.c_double), ("ms_solve", C.c_double),
                ("ms_linesearch", C.c_double), ("ms_pf", C.c_double), ("graph_iters", C.c_int),
                ("soc_steps", C.c_int), ("restorations", C.c_int), ("resto_iters", C.c_int)]


OPF_LINRED, OPF_REDLIN = 0, 1

# name -> (restype, argtypes)
_SIGS = {
    "opf_create": (C.c_int, [C.POINTER(opf_network), C.POINTER(opf_options), C.POINTER(C.c_void_p)]),
    "opf_destroy": (None, [C.c_void_p]),
    "opf_strerror": (C.c_char_p, [C.c_int]),
    "opf_sizes": (C.c_int, [C.c_void_p, _ip, _ip, _ip]),
    "opf_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), _ip, _ip, C.POINTER(C.c_longlong),
                            C.POINTER(C.c_longlong)]),
    "opf_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "opf_trsm_choice": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_float), _ip]),
    "opf_chol_choice": (C.c_int, [C.c_void_p, _ip, _ip, C.POINTER(C.c_float)]),
    "opf_chol_solve_choice": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_float)]),
    "opf_forward_reach": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_double)]),
    "opf_route_choice": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_float)]),
    "opf_rhs_width": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_float)]),
    "opf_eval_derivatives": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_eval_functions": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_get_vector": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "opf_get_csr_pattern": (C.c_int, [C.c_void_p, C.c_int, _ip, _ip, C.POINTER(C.c_longlong), C.c_void_p,
                                      C.c_void_p]),
    "opf_get_csr_values": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "opf_gx_factor": (C.c_int, [C.c_void_p]),
    "opf_gx_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "opf_condense": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_kkt_factor": (C.c_int, [C.c_void_p, C.c_double, C.c_double, _ip]),
    "opf_get_factor": (C.c_int, [C.c_void_p, C.c_void_p]),
    "opf_newton_step": (C.c_int, [C.c_void_p] + [C.c_void_p] * 8 + [C.c_double, C.c_double, C.c_void_p, _ip]),
    "opf_kkt_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "opf_condense_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_kkt_solve_condensed": (C.c_int, [C.c_void_p, C.c_void_p]),
    "opf_kkt_solve_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "opf_fullspace_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                       _ip]),
    "opf_fullspace_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, _ip,
                                      C.POINTER(C.c_double)]),
    "opf_fullspace_stats": (C.c_int, [C.c_void_p, _ip, _ip, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double), _ip]),
    "opf_fullspace_tuning": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_float)]),
    "opf_powerflow": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, _ip]),
    "opf_reduced_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_solve": (C.c_int, [C.c_void_p, C.POINTER(opf_ipm_options), C.POINTER(opf_ipm_result)]),
    "opf_get_solution": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_set_loads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_vjp_prepare": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "opf_dispatch_vjp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "opf_vjp_info": (C.c_int, [C.c_void_p, _ip, C.POINTER(C.c_double), _ip, C.POINTER(C.c_double)]),
    "opf_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "opf_batch_destroy": (None, [C.c_void_p]),
    "opf_batch_size": (C.c_int, [C.c_void_p, _ip, _ip]),
    "opf_batch_autotune": (C.c_int, [C.c_void_p]),
    "opf_batch_solve": (C.c_int, [C.c_void_p, C.POINTER(opf_ipm_options), C.POINTER(opf_ipm_result),
                                  C.POINTER(C.c_double)]),
    "opf_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "opf_batch_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), _ip, _ip, C.POINTER(C.c_float),
                                  C.POINTER(C.c_longlong)]),
    "opf_batch_condense_factor": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                            C.POINTER(C.c_void_p), C.POINTER(C.c_double), _ip, _ip]),
    "opf_chol_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, _ip, C.c_void_p]),
    "opf_launch_count": (C.c_ulonglong, []),
    "opf_fp64_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "opf_last_cuda_error": (C.c_int, [C.c_char_p, C.c_int]),
    "opf_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "opf_phase_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
}

PHASES = ("refactor", "assemble", "trsm", "spmm", "kred", "chol", "rhs", "recover")

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libcondipm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2203_11875_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def launch_count() -> int:
    """Kernel launches libcondipm.so has enqueued since it was loaded."""
    return int(load_library().opf_launch_count())


def fp64_peak(which: int = 0) -> float:
    """opf_fp64_peak: measured FP64 GFLOP/s of the current device (0 DFMA,
    1/2/3 mma.sync f64 m8n8k4 / m16n8k4 / m16n8k16)."""
    g = C.c_double(0.0)
    _check(load_library().opf_fp64_peak(int(which), C.byref(g)), "opf_fp64_peak")
    return g.value


def chol_noalloc(A, n, delta_w, L, stream=None):
    """opf_chol_noalloc: factor A + delta_w I = L L^T (device n x n buffers) with no
    device allocation.  Returns -1 on success, else the failing column."""
    col = C.c_int(-1)
    rc = load_library().opf_chol_noalloc(_ptr(A), int(n), float(delta_w), _ptr(L), C.byref(col),
                                         None if stream is None else C.c_void_p(stream.cuda_stream))
    if rc == OPF_ERR_NOT_PD:
        return col.value
    _check(rc, "opf_chol_noalloc")
    return -1


class OPFError(RuntimeError):
    def __init__(self, code: int, where: str, info: int = -1):
        self.code = code
        self.info = info
        lib = load_library()
        msg = lib.opf_strerror(code).decode()
        if code == -2:
            buf = C.create_string_buffer(64)
            e = lib.opf_last_cuda_error(buf, 64)
            msg += f" [{buf.value.decode()} ({e})]"
        super().__init__(f"{where}: {msg} (status {code})")


def _check(code: int, where: str):
    if code != OPF_OK:
        raise OPFError(code, where)


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or t.dtype.itemsize != 8 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _host_ptr(a, writable=False):
    """Host pointer of a contiguous float64 CPU tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or (writable and not a.flags.writeable):
            raise ValueError("expected a contiguous float64 numpy array")
        return C.c_void_p(a.ctypes.data)
    if getattr(a, "is_cuda", True) or a.dtype.itemsize != 8 or not a.is_contiguous():
        raise ValueError("expected a contiguous float64 CPU tensor")
    return C.c_void_p(a.data_ptr())


class Handle:
    """One network on one GPU: wraps opf_create / opf_destroy and every call."""

    def __init__(self, net, route: int = OPF_ROUTE_ADJOINT, rhs_block: int = 0, spin_limit: int = 0,
                 chol_form: int = 0, rhs1_kernel: int = 0, rhs_width: int = 0, dense_forward: int = 0):
        lib = load_library()
        self._keep = []

        def d(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(_dp)

        def i(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self._keep.append(a)
            return a.ctypes.data_as(_ip)
        n = opf_network(net.nb, net.nl, net.ng, net.slack, d(net.Pd), d(net.Qd), d(net.Vmin), d(net.Vmax),
                        i(net.lf), i(net.lt), d(net.r), d(net.x), d(net.b), d(net.rate), i(net.gbus),
                        d(net.Pmin), d(net.Pmax), d(net.Qmin), d(net.Qmax), d(net.c2), d(net.c1))
        o = opf_options(route, rhs_block, spin_limit, chol_form, rhs1_kernel, rhs_width, dense_forward)
        h = C.c_void_p()
        _check(lib.opf_create(C.byref(n), C.byref(o), C.byref(h)), "opf_create")
        self._keep = []
        self._h = h
        self._lib = lib
        nx, nu, m = C.c_int(), C.c_int(), C.c_int()
        _check(lib.opf_sizes(h, C.byref(nx), C.byref(nu), C.byref(m)), "opf_sizes")
        self.nx, self.nu, self.m = nx.value, nu.value, m.value
        self.nw = self.nx + self.nu
        self.nb, self.ng = int(net.nb), int(net.ng)
        self.n_kkt = self.nw + 2 * self.m + self.nx

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.opf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- ABI calls (same names as the C entry points, without the opf_ prefix)
    def stats(self):
        a, b, c, d_, e = C.c_longlong(), C.c_int(), C.c_int(), C.c_longlong(), C.c_longlong()
        _check(self._lib.opf_stats(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d_), C.byref(e)),
               "opf_stats")
        return dict(nnz_lu=a.value, levels_fwd=b.value, levels_bwd=c.value, nnz_k=d_.value,
                    lu_flops=e.value)

    def trsm_choice(self):
        """(multi-RHS kernel, autotuner ms per candidate, single-RHS kernel)."""
        k, k1 = C.c_int(), C.c_int()
        ms = (C.c_float * 6)()
        _check(self._lib.opf_trsm_choice(self._h, C.byref(k), ms, C.byref(k1)), "opf_trsm_choice")
        names = ("cols", "staged1", "staged2", "staged4", "blocked", "dataflow")
        return k.value, dict(zip(names, ms)), k1.value

    def chol_choice(self):
        """(Cholesky form: 1 barrier, 2 dataflow, 0 not tuned yet; its grid;
        autotuner ms per candidate)."""
        f, nb = C.c_int(), C.c_int()
        ms = (C.c_float * 11)()
        _check(self._lib.opf_chol_choice(self._h, C.byref(f), C.byref(nb), ms), "opf_chol_choice")
        names = ("barrier_quarter_sm", "barrier_half_sm", "barrier_1_per_sm", "barrier_2_per_sm",
                 "dataflow_half_sm", "dataflow_1_per_sm", "dataflow_2_per_sm", "dataflow_1_per_sm_wide_panel",
                 "dataflow_2_per_sm_wide_panel", "dataflow_4_per_sm", "dataflow_4_per_sm_wide_panel")
        return f.value, nb.value, dict(zip(names, ms))

    def chol_solve_choice(self):
        """(cluster size of the few-right-hand-side dense solve; {4, 8, 16: ms}
        of its timing on the first one-vector solve, 0 = not timed)."""
        c = C.c_int()
        ms = (C.c_float * 3)()
        _check(self._lib.opf_chol_solve_choice(self._h, C.byref(c), ms), "opf_chol_solve_choice")
        return c.value, dict(zip((4, 8, 16), ms))

    def forward_reach(self):
        """(32-column blocks of the forward sweep with a reach list; {"listed":
        multiply-adds of their listed rows, "all": of all their rows})."""
        nb = C.c_int()
        wk = (C.c_double * 2)()
        _check(self._lib.opf_forward_reach(self._h, C.byref(nb), wk), "opf_forward_reach")
        return nb.value, {"listed": wk[0], "all": wk[1]}

    def route_choice(self):
        """(route in use: 0 adjoint, 1 explicit, -1 auto before its first
        condensation; {"adjoint": ms, "explicit": ms} of the AUTO timing)."""
        r = C.c_int()
        ms = (C.c_float * 2)()
        _check(self._lib.opf_route_choice(self._h, C.byref(r), ms), "opf_route_choice")
        return r.value, {"adjoint": ms[0], "explicit": ms[1]}

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream (or None for the legacy default stream)."""
        ptr = None if stream is None else C.c_void_p(stream.cuda_stream)
        _check(self._lib.opf_set_stream(self._h, ptr), "opf_set_stream")

    def eval_derivatives(self, x, u, lam=None, y=None):
        _check(self._lib.opf_eval_derivatives(self._h, _ptr(x), _ptr(u), _ptr(lam), _ptr(y)),
               "opf_eval_derivatives")

    def eval_functions(self, x, u):
        _check(self._lib.opf_eval_functions(self._h, _ptr(x), _ptr(u)), "opf_eval_functions")

    def get_vector(self, which, dst):
        _check(self._lib.opf_get_vector(self._h, which, _ptr(dst)), "opf_get_vector")

    def get_csr_pattern(self, which):
        nr, nc, nnz = C.c_int(), C.c_int(), C.c_longlong()
        _check(self._lib.opf_get_csr_pattern(self._h, which, C.byref(nr), C.byref(nc), C.byref(nnz), None,
                                             None), "opf_get_csr_pattern")
        rp = np.zeros(nr.value + 1, np.int32)
        ci = np.zeros(max(1, nnz.value), np.int32)
        _check(self._lib.opf_get_csr_pattern(self._h, which, None, None, None, rp.ctypes.data_as(C.c_void_p),
                                             ci.ctypes.data_as(C.c_void_p)), "opf_get_csr_pattern")
        return nr.value, nc.value, rp, ci[:nnz.value]

    def get_csr_values(self, which, dst):
        _check(self._lib.opf_get_csr_values(self._h, which, _ptr(dst)), "opf_get_csr_values")

    def gx_factor(self):
        _check(self._lib.opf_gx_factor(self._h), "opf_gx_factor")

    def gx_solve(self, trans, B, X, nrhs=1):
        _check(self._lib.opf_gx_solve(self._h, int(trans), _ptr(B), _ptr(X), int(nrhs)), "opf_gx_solve")

    def condense(self, sig_u, sig_x, sig_s, Kred=None):
        _check(self._lib.opf_condense(self._h, _ptr(sig_u), _ptr(sig_x), _ptr(sig_s), _ptr(Kred)),
               "opf_condense")

    def kkt_factor(self, delta_w=0.0, delta_c=0.0):
        """Returns -1 on success, else the failing column (status NOT_PD)."""
        col = C.c_int(-1)
        rc = self._lib.opf_kkt_factor(self._h, float(delta_w), float(delta_c), C.byref(col))
        if rc == OPF_ERR_NOT_PD:
            return col.value
        _check(rc, "opf_kkt_factor")
        return -1

    def newton_step(self, x, u, lam, y, sig_u, sig_x, sig_s, rhs, step, delta_w=0.0, delta_c=0.0):
        """opf_newton_step with HOST buffers: float64 CPU tensors or numpy arrays
        (contiguous; pinned tensors make the copies asynchronous).  Returns -1
        on success, else the failing Cholesky column (no step written)."""
        args = [_host_ptr(a) for a in (x, u, lam, y, sig_u, sig_x, sig_s, rhs)]
        col = C.c_int(-1)
        rc = self._lib.opf_newton_step(self._h, *args, float(delta_w), float(delta_c), _host_ptr(step, True),
                                       C.byref(col))
        if rc == OPF_ERR_NOT_PD:
            return col.value
        _check(rc, "opf_newton_step")
        return -1

    def get_factor(self, dst):
        _check(self._lib.opf_get_factor(self._h, _ptr(dst)), "opf_get_factor")

    def condense_rhs(self, sig_u, sig_x, sig_s, rhs, Kred=None):
        _check(self._lib.opf_condense_rhs(self._h, _ptr(sig_u), _ptr(sig_x), _ptr(sig_s), _ptr(rhs), _ptr(Kred)),
               "opf_condense_rhs")

    def kkt_solve_condensed(self, step):
        _check(self._lib.opf_kkt_solve_condensed(self._h, _ptr(step)), "opf_kkt_solve_condensed")

    def kkt_solve(self, rhs, step, nrhs=1):
        _check(self._lib.opf_kkt_solve(self._h, _ptr(rhs), _ptr(step), int(nrhs)), "opf_kkt_solve")

    def kkt_solve_adjoint(self, rhs, sol, nrhs=1):
        _check(self._lib.opf_kkt_solve_adjoint(self._h, _ptr(rhs), _ptr(sol), int(nrhs)),
               "opf_kkt_solve_adjoint")

    def fullspace_factor(self, sig_u, sig_x, sig_s, delta_w=0.0, delta_c=0.0):
        """opf_fullspace_factor: returns (status, (n+, n-, n0)); status is OPF_OK
        or OPF_ERR_NOT_PD (wrong inertia), other codes raise."""
        inert = (C.c_int * 3)()
        rc = self._lib.opf_fullspace_factor(self._h, _ptr(sig_u), _ptr(sig_x), _ptr(sig_s), float(delta_w),
                                            float(delta_c), inert)
        if rc not in (OPF_OK, OPF_ERR_NOT_PD):
            _check(rc, "opf_fullspace_factor")
        return rc, tuple(inert)

    def fullspace_solve(self, rhs, step, nrhs=1, refine=0):
        """opf_fullspace_solve: returns (corrections taken, final relative residual)."""
        st = C.c_int(0)
        res = C.c_double(0.0)
        _check(self._lib.opf_fullspace_solve(self._h, _ptr(rhs), _ptr(step), int(nrhs), int(refine), C.byref(st),
                                             C.byref(res)), "opf_fullspace_solve")
        return st.value, res.value

    def fullspace_stats(self):
        nb, lv = C.c_int(0), C.c_int(0)
        nl, fl = C.c_longlong(0), C.c_longlong(0)
        ld = C.c_double(0.0)
        inert = (C.c_int * 3)()
        _check(self._lib.opf_fullspace_stats(self._h, C.byref(nb), C.byref(lv), C.byref(nl), C.byref(fl),
                                             C.byref(ld), inert), "opf_fullspace_stats")
        return dict(nblocks=nb.value, levels=lv.value, nnz_l=nl.value, flops=fl.value, logabsdet=ld.value,
                    inertia=tuple(inert))

    def rhs_width(self):
        """opf_rhs_width: (N in use, autotuner timings at nu, 512, 256, 128)."""
        w = C.c_int(0)
        ms = (C.c_float * 4)()
        _check(self._lib.opf_rhs_width(self._h, C.byref(w), ms), "opf_rhs_width")
        return w.value, list(ms)

    def fullspace_tuning(self):
        g = (C.c_int * 2)()
        ms = (C.c_float * 8)()
        _check(self._lib.opf_fullspace_tuning(self._h, g, ms), "opf_fullspace_tuning")
        return dict(grid_factor=g[0], grid_solve=g[1], factor_ms=list(ms[:4]), solve_ms=list(ms[4:]))

    def solve(self, variant="linred", tol=1e-8, max_iter=300, mu0=0.1, pf_tol=1e-10, verbose=False,
              line_search="merit", linear_solver="condensed", restoration=False, start_with_resto=False):
        """opf_solve: the interior-point loop; returns the result fields as a dict.
        line_search: "merit" or "filter" (LinRed); linear_solver: "condensed" or
        "fullspace" (the hybrid full-space IPM, LinRed); restoration /
        start_with_resto: the feasibility restoration phase of the filter line
        search."""
        o = _ipm_options(variant, tol, max_iter, mu0, pf_tol, verbose, line_search, linear_solver, restoration,
                         start_with_resto)
        r = opf_ipm_result()
        rc = self._lib.opf_solve(self._h, C.byref(o), C.byref(r))
        out = {f: getattr(r, f) for f, _ in opf_ipm_result._fields_}
        self.last_result = out
        if rc not in (OPF_OK, OPF_ERR_NO_CONVERGENCE, OPF_ERR_INFEASIBLE):
            raise OPFError(rc, "opf_solve")
        return out

    def solution(self):
        """(w = [u; x], lam, y, Pg) of the last solve, host numpy arrays."""
        w = np.zeros(self.nw)
        lam = np.zeros(self.nx)
        y = np.zeros(self.m)
        pg = np.zeros((self.nu + 1) // 2)
        _check(self._lib.opf_get_solution(self._h, w.ctypes.data_as(C.c_void_p), lam.ctypes.data_as(C.c_void_p),
                                          y.ctypes.data_as(C.c_void_p), pg.ctypes.data_as(C.c_void_p)),
               "opf_get_solution")
        return w, lam, y, pg

    def set_loads(self, Pd, Qd):
        """opf_set_loads: host arrays of nb loads (the library copies them)."""
        Pd = np.ascontiguousarray(Pd, dtype=np.float64)
        Qd = np.ascontiguousarray(Qd, dtype=np.float64)
        if Pd.shape != (self.nb,) or Qd.shape != (self.nb,):
            raise ValueError(f"expected Pd, Qd of shape ({self.nb},)")
        _check(self._lib.opf_set_loads(self._h, Pd.ctypes.data_as(C.c_void_p), Qd.ctypes.data_as(C.c_void_p)),
               "opf_set_loads")

    def vjp_prepare(self, w=None, lam=None, y=None, sig_w=None, sig_s=None):
        """opf_vjp_prepare: factor K_aug at the given point (host arrays) or, with
        no arguments, at the last solve's solution."""
        args = [w, lam, y, sig_w, sig_s]
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in args]
        ptrs = [None if a is None else a.ctypes.data_as(C.c_void_p) for a in keep]
        _check(self._lib.opf_vjp_prepare(self._h, *ptrs), "opf_vjp_prepare")

    def dispatch_vjp(self, vbar, grad_Pd, grad_Qd):
        """opf_dispatch_vjp: vbar (k, ng) -> grad_Pd, grad_Qd (k, nb), device tensors."""
        k = 0 if vbar.numel() == 0 else vbar.shape[0]
        _check(self._lib.opf_dispatch_vjp(self._h, _ptr(vbar), int(k), _ptr(grad_Pd), _ptr(grad_Qd)),
               "opf_dispatch_vjp")

    def vjp_info(self):
        """dict: refinement corrections and relative residual of the last
        dispatch_vjp; Newton iterations and KKT residual of the last polish."""
        n, r, pi, pr = C.c_int(), C.c_double(), C.c_int(), C.c_double()
        _check(self._lib.opf_vjp_info(self._h, C.byref(n), C.byref(r), C.byref(pi), C.byref(pr)), "opf_vjp_info")
        return dict(refine_steps=n.value, rel_residual=r.value, polish_iters=pi.value, kkt_residual=pr.value)

    def profile(self, enable=True):
        _check(self._lib.opf_profile(self._h, int(bool(enable))), "opf_profile")

    def phase_times(self):
        ms = (C.c_double * len(PHASES))()
        n = (C.c_longlong * len(PHASES))()
        _check(self._lib.opf_phase_times(self._h, ms, n), "opf_phase_times")
        return {p: (ms[i], n[i]) for i, p in enumerate(PHASES)}

    def reduced_gradient(self, grad, grad_r, lam=None):
        """opf_reduced_gradient: grad (nu+nx device vector, or None for grad f) ->
        grad_r (nu) and, when given, the adjoint lam (nx)."""
        _check(self._lib.opf_reduced_gradient(self._h, _ptr(grad), _ptr(grad_r), _ptr(lam)),
               "opf_reduced_gradient")

    def powerflow(self, u, x, tol=1e-10, max_iter=30):
        it = C.c_int(0)
        _check(self._lib.opf_powerflow(self._h, _ptr(u), _ptr(x), float(tol), int(max_iter), C.byref(it)),
               "opf_powerflow")
        return it.value


def _ipm_options(variant="linred", tol=1e-8, max_iter=300, mu0=0.1, pf_tol=1e-10, verbose=False,
                 line_search="merit", linear_solver="condensed", restoration=False, start_with_resto=False):
    if linear_solver not in ("condensed", "fullspace"):
        raise ValueError(f"linear_solver: {linear_solver!r}")
    return opf_ipm_options(OPF_LINRED if variant == "linred" else OPF_REDLIN, tol, max_iter, mu0, pf_tol,
                           int(bool(verbose)), 1 if line_search == "filter" else 0, int(bool(restoration)),
                           int(bool(start_with_resto)), 1 if linear_solver == "fullspace" else 0)


class Batch:
    """Concurrent interior-point solves of several handles (opf_batch_*)."""

    def __init__(self, handles, nthreads: int = 0):
        lib = load_library()
        self._handles = list(handles)      # keeps the handles alive while the batch lives
        arr = (C.c_void_p * len(self._handles))(*[h._h.value for h in self._handles])
        b = C.c_void_p()
        _check(lib.opf_batch_create(arr, len(self._handles), int(nthreads), C.byref(b)), "opf_batch_create")
        self._b, self._lib = b, lib
        n, t = C.c_int(), C.c_int()
        _check(lib.opf_batch_size(b, C.byref(n), C.byref(t)), "opf_batch_size")
        self.n, self.nthreads = n.value, t.value

    def autotune(self):
        _check(self._lib.opf_batch_autotune(self._b), "opf_batch_autotune")

    def solve(self, **options):
        """opf_batch_solve; returns (per-instance result dicts, host wall ms)."""
        o = _ipm_options(**options)
        res = (opf_ipm_result * self.n)()
        ms = C.c_double()
        rc = self._lib.opf_batch_solve(self._b, C.byref(o), res, C.byref(ms))
        out = [{f: getattr(r, f) for f, _ in opf_ipm_result._fields_} for r in res]
        if rc not in (OPF_OK, OPF_ERR_NO_CONVERGENCE, OPF_ERR_INFEASIBLE):
            raise OPFError(rc, "opf_batch_solve")
        return out, ms.value

    def set_mode(self, mode):
        """opf_batch_set_mode: "lockstep" (batched condensation every iteration)
        or "concurrent" (independent loops on streams)."""
        code = {"concurrent": 0, "lockstep": 1}[mode]
        _check(self._lib.opf_batch_set_mode(self._b, code), "opf_batch_set_mode")

    def lockstep_calls(self):
        return self.stats()["lockstep_calls"]

    def stats(self):
        """opf_batch_stats: lockstep condensations, the batched solve's and
        Cholesky's cluster sizes and their tuning timings."""
        n, a, c, g = C.c_longlong(0), C.c_int(0), C.c_int(0), C.c_longlong(0)
        ms = (C.c_float * 8)()
        _check(self._lib.opf_batch_stats(self._b, C.byref(n), C.byref(a), C.byref(c), ms, C.byref(g)),
               "opf_batch_stats")
        return dict(lockstep_calls=n.value, trsm_cl=a.value, chol_cl=c.value,
                    tune_trsm_ms=list(ms[:4]), tune_chol_ms=list(ms[4:]), graph_calls=g.value)

    def condense_factor(self, sig_u, sig_x, sig_s, delta_w=None):
        """opf_batch_condense_factor: per-instance device tensors of Sigma (lists
        of n tensors) and delta_w (n floats or None).  Returns (status list,
        failing-column list)."""
        n = self.n
        if not (len(sig_u) == len(sig_x) == len(sig_s) == n):
            raise ValueError(f"expected {n} tensors per Sigma block")
        arr = [(C.c_void_p * n)(*[_ptr(t).value for t in blk]) for blk in (sig_u, sig_x, sig_s)]
        dw = None if delta_w is None else (C.c_double * n)(*[float(v) for v in delta_w])
        st = (C.c_int * n)()
        fc = (C.c_int * n)()
        rc = self._lib.opf_batch_condense_factor(self._b, arr[0], arr[1], arr[2], dw, st, fc)
        if rc not in (OPF_OK, OPF_ERR_NOT_PD, OPF_ERR_SINGULAR, OPF_ERR_TIMEOUT):
            raise OPFError(rc, "opf_batch_condense_factor")
        return list(st), list(fc)

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.opf_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
