"""ctypes binding of the C ABI in include/topo.h (argument marshalling only).

Device arrays are torch CUDA tensors (FP64, contiguous); every computation runs in the CUDA
library.  Importing this module loads ``libtopo_gb300.so`` and raises ImportError if it has not
been built (``python -m paper_1606_06201_gb300.build``): there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TOPO_LIBRARY: another build of the library (e.g. the index-checked libtopo_gb300_bc.so)
LIB_PATH = os.environ.get("TOPO_LIBRARY") or os.path.join(_HERE, "libtopo_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("%s is missing: build it with "
                      "`python -m paper_1606_06201_gb300.build` (nvcc, sm_103a)" % LIB_PATH)
_lib = ctypes.CDLL(LIB_PATH)

OK, E_INVALID_ARG, E_NOT_CONVERGED, E_BREAKDOWN, E_INFEASIBLE, E_TIMEOUT, E_OOM, E_CUDA, E_BOUNDS = \
    range(9)
FP64, MIXED = 0, 1
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_CONVERGED", 3: "BREAKDOWN", 4: "INFEASIBLE",
                5: "TIMEOUT", 6: "OOM", 7: "CUDA", 8: "BOUNDS"}


class SolverDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("fixed", ctypes.POINTER(ctypes.c_uint8)), ("levels", ctypes.c_int),
                ("precision", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("max_iter", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("flexible", ctypes.c_int), ("generic_kernels", ctypes.c_int),
                ("smoother", ctypes.c_int), ("omega_auto", ctypes.c_int),
                ("K0", ctypes.POINTER(ctypes.c_double))]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("status", ctypes.c_int)]


class IpOpts(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("tau_nwt", ctypes.c_double),
                ("tau_ip", ctypes.c_double), ("frac", ctypes.c_double),
                ("step_x_only", ctypes.c_int), ("max_newton", ctypes.c_int),
                ("cg_tol", ctypes.c_double), ("cg_tol_init", ctypes.c_double),
                ("cg_tol_factor", ctypes.c_double), ("stop_rule", ctypes.c_int),
                ("tau_kkt", ctypes.c_double)]


class IpInfo(ctypes.Structure):
    _fields_ = [("newton", ctypes.c_int), ("ip_iters", ctypes.c_int), ("feval", ctypes.c_int),
                ("cg_iters", ctypes.c_int), ("s", ctypes.c_double), ("r", ctypes.c_double),
                ("lam", ctypes.c_double), ("alpha", ctypes.c_double), ("crit", ctypes.c_double),
                ("done", ctypes.c_int), ("status", ctypes.c_int), ("wall_ms", ctypes.c_double),
                ("kkt", ctypes.c_double)]


class OcOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("q", ctypes.c_double), ("xlow", ctypes.c_double),
                ("lam_hi", ctypes.c_double), ("tau_lambda", ctypes.c_double),
                ("tau_oc", ctypes.c_double), ("max_feval", ctypes.c_int),
                ("cg_tol0", ctypes.c_double), ("adaptive_tol", ctypes.c_int)]


class OcInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("feval", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("compliance", ctypes.c_double), ("compliance_prev", ctypes.c_double),
                ("lam", ctypes.c_double), ("cg_tol", ctypes.c_double), ("status", ctypes.c_int),
                ("wall_ms", ctypes.c_double)]


OC_PLAIN, OC_DOC, OC_AOC = 0, 1, 2

_vp = ctypes.c_void_p
_SIGS = {
    "topo_last_error": (ctypes.c_char_p, []),
    "topo_element_stiffness": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp]),
    "topo_solver_create": (ctypes.c_int, [ctypes.POINTER(SolverDesc), ctypes.POINTER(_vp)]),
    "topo_solver_destroy": (ctypes.c_int, [_vp]),
    "topo_set_stream": (ctypes.c_int, [_vp, _vp]),
    "topo_set_graph_mode": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_set_vcycle_fusion": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_set_outer_precision": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_set_profiling_mask": (ctypes.c_int, [_vp, ctypes.c_uint]),
    "topo_get_profile_kernel": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_longlong)]),
    "topo_solver_device_bytes": (ctypes.c_size_t, [_vp]),
    "topo_solver_launch_count": (ctypes.c_ulonglong, [_vp]),
    "topo_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_get_profile": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_longlong)]),
    "topo_set_density": (ctypes.c_int, [_vp, _vp]),
    "topo_solve_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, _vp]),
    "topo_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(SolveInfo)]),
    "topo_apply_K": (ctypes.c_int, [_vp, _vp, _vp]),
    "topo_apply_vcycle": (ctypes.c_int, [_vp, _vp, _vp]),
    "topo_check_conversions": (ctypes.c_int, [_vp, _vp, ctypes.c_longlong, _vp]),
    "topo_bounds_check_enabled": (ctypes.c_int, []),
    "topo_bounds_report": (ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong),
                                          ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_longlong), ctypes.c_char_p,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "topo_bounds_selftest": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_longlong]),
    "topo_get_level_matrices": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "topo_level_elems": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_compliance": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "topo_element_energy": (ctypes.c_int, [_vp, _vp, _vp]),
    "topo_grad_x": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "topo_compliance_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_longlong, ctypes.c_int, _vp,
                                               _vp]),
    "topo_ip_create": (ctypes.c_int, [ctypes.POINTER(SolverDesc), _vp, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(_vp)]),
    "topo_ip_destroy": (ctypes.c_int, [_vp]),
    "topo_ip_set_stream": (ctypes.c_int, [_vp, _vp]),
    "topo_ip_init": (ctypes.c_int, [_vp, ctypes.POINTER(IpOpts)]),
    "topo_ip_step": (ctypes.c_int, [_vp, ctypes.POINTER(IpOpts), ctypes.POINTER(IpInfo)]),
    "topo_ip_run": (ctypes.c_int, [_vp, ctypes.POINTER(IpOpts), ctypes.POINTER(IpInfo)]),
    "topo_ip_get_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "topo_ip_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "topo_ip_power_state_size": (ctypes.c_int, [_vp, _vp]),
    "topo_ip_set_vcycle_fusion": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_ip_set_simp": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
    "topo_ip_filtered_density": (ctypes.c_int, [_vp, _vp]),
    "topo_ip_get_power_state": (ctypes.c_int, [_vp, _vp, _vp]),
    "topo_ip_set_power_state": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "topo_oc_create": (ctypes.c_int, [ctypes.POINTER(SolverDesc), _vp, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(_vp)]),
    "topo_oc_destroy": (ctypes.c_int, [_vp]),
    "topo_oc_set_stream": (ctypes.c_int, [_vp, _vp]),
    "topo_oc_init": (ctypes.c_int, [_vp, _vp]),
    "topo_oc_step": (ctypes.c_int, [_vp, ctypes.POINTER(OcOpts), ctypes.POINTER(OcInfo)]),
    "topo_oc_run": (ctypes.c_int, [_vp, ctypes.POINTER(OcOpts), ctypes.POINTER(OcInfo)]),
    "topo_oc_get_x": (ctypes.c_int, [_vp, _vp]),
    "topo_oc_get_u": (ctypes.c_int, [_vp, _vp]),
    "topo_oc_get_state": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "topo_oc_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "topo_oc_power_state_size": (ctypes.c_int, [_vp, _vp]),
    "topo_oc_get_power_state": (ctypes.c_int, [_vp, _vp, _vp]),
    "topo_oc_set_power_state": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "topo_solver_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(SolverDesc),
                                                   ctypes.POINTER(ctypes.c_size_t)]),
    "topo_set_record_file": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "topo_set_sweep_rows": (ctypes.c_int, [_vp, ctypes.c_int]),
    "topo_set_wait_limit_ns": (ctypes.c_int, [_vp, ctypes.c_ulonglong]),
    "topo_ip_set_record_file": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "topo_oc_set_record_file": (ctypes.c_int, [_vp, ctypes.c_char_p]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class TopoError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.topo_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))
        self.status = status


def _check(status, where, allow=()):
    if status != OK and status not in allow:
        raise TopoError(status, where)
    return status


def _torch_f64():
    import torch
    return torch.float64


def _ptr(t):
    """Device pointer of a contiguous FP64 CUDA tensor."""
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def element_stiffness(dim, E=1.0, nu=0.3):
    ne = 8 if dim == 2 else 24
    K0 = np.zeros((ne, ne))
    _check(_lib.topo_element_stiffness(dim, E, nu, K0.ctypes.data_as(_vp)), "topo_element_stiffness")
    return K0


JACOBI, CHEBYSHEV = 0, 1


def _k0_array(dim, K0):
    """The caller's element matrix as a contiguous FP64 host array (None: the analytic K0)."""
    if K0 is None:
        return None
    ne = 8 if dim == 2 else 24
    a = np.ascontiguousarray(np.asarray(K0, dtype=np.float64))
    if a.size != ne * ne:
        raise ValueError("K0 has %d entries, expected %d" % (a.size, ne * ne))
    return a


def _desc(nx, ny, nz, fixed, levels, precision, nu1, nu2, omega, max_iter, nrhs, flexible, E, nu,
          generic_kernels, omega_auto=False, smoother=0, K0=None):
    dim = 3 if nz else 2
    n = dim * (nx + 1) * (ny + 1) * ((nz + 1) if nz else 1)
    if fixed is None:
        fixed = np.zeros(n, dtype=np.uint8)
    fixed = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
    if fixed.size != n:
        raise ValueError("fixed mask has %d entries, expected %d" % (fixed.size, n))
    if omega is None:
        omega = 0.6 if dim == 2 else 0.5
    if flexible is None:
        flexible = 0
    k0 = _k0_array(dim, K0)
    d = SolverDesc(dim, nx, ny, nz, E, nu, fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                   levels, precision, nu1, nu2, omega, max_iter, nrhs, flexible,
                   int(generic_kernels), int(smoother), int(omega_auto),
                   None if k0 is None else k0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    d._keep = (fixed, k0)  # the host arrays must outlive the create call
    return d, fixed, dim, n


def workspace_bytes(nx, ny, nz=0, fixed=None, levels=3, precision=FP64, nu1=2, nu2=2, omega=None,
                    max_iter=1000, nrhs=1, flexible=None, E=1.0, nu=0.3, generic_kernels=False,
                    omega_auto=False, smoother=0, K0=None):
    """Device bytes a Solver with these arguments allocates (topo_solver_workspace_bytes)."""
    d, _, _, _ = _desc(nx, ny, nz, fixed, levels, precision, nu1, nu2, omega, max_iter, nrhs,
                       flexible, E, nu, generic_kernels, omega_auto, smoother, K0)
    out = ctypes.c_size_t(0)
    _check(_lib.topo_solver_workspace_bytes(ctypes.byref(d), ctypes.byref(out)),
           "topo_solver_workspace_bytes")
    return int(out.value)


def ip_options(sigma=0.2, tau_nwt=0.1, tau_ip=1e-8, frac=0.9, step_x_only=False, max_newton=500,
               cg_tol=1e-8, cg_tol_init=None, cg_tol_factor=1.0, stop_rule="barrier",
               tau_kkt=1e-6):
    """Sec. 3 defaults; cg_tol is the relative residual of the Z solves of the first major
    iteration, multiplied by cg_tol_factor at every barrier reduction (Sec. 8.1: 1e-2 with factor
    1 or 0.5).  stop_rule "barrier" (max(s, r) <= tau_ip) or "kkt" (the scaled KKT residual of
    the Remark in Sec. 3.4 <= tau_kkt)."""
    if stop_rule not in ("barrier", "kkt"):
        raise ValueError("stop_rule must be 'barrier' or 'kkt'")
    return IpOpts(sigma, tau_nwt, tau_ip, frac, int(step_x_only), max_newton, cg_tol,
                  cg_tol if cg_tol_init is None else cg_tol_init, cg_tol_factor,
                  0 if stop_rule == "barrier" else 1, tau_kkt)


def oc_options(variant=OC_AOC, q=0.5, xlow=1e-6, lam_hi=1e4, tau_lambda=1e-11, tau_oc=1e-5,
               max_feval=10000, cg_tol0=1e-4, adaptive_tol=True):
    """Sec. 4 and Sec. 6.2 defaults."""
    return OcOpts(variant, q, xlow, lam_hi, tau_lambda, tau_oc, max_feval, cg_tol0,
                  int(adaptive_tol))



def bounds_check_enabled():
    """True when the loaded library is the index-checked build (TOPO_BOUNDS_CHECK)."""
    return bool(_lib.topo_bounds_check_enabled())


def bounds_report(reset=False):
    """(count, first index, its size, file, line) of the index checks of the debug build."""
    count, index, size, line = ctypes.c_ulonglong(), ctypes.c_longlong(), ctypes.c_longlong(), \
        ctypes.c_int()
    buf = ctypes.create_string_buffer(512)
    _check(_lib.topo_bounds_report(ctypes.byref(count), ctypes.byref(index), ctypes.byref(size),
                                   buf, 512, ctypes.byref(line), int(reset)), "topo_bounds_report")
    return count.value, index.value, size.value, buf.value.decode(), line.value


def bounds_selftest(i, n):
    """One index check of i against n in a kernel that addresses no buffer (debug build)."""
    _check(_lib.topo_bounds_selftest(int(i), int(n)), "topo_bounds_selftest")


def check_conversions(d, f):
    """Mismatch counts (double -> float, float -> double) of the library's integer conversions
    against the hardware ones on the entries of d (FP64 CUDA tensor) and f (FP32 CUDA tensor of
    the same length)."""
    import torch
    if d.numel() != f.numel():
        raise ValueError("d and f must have the same length")
    if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    out = (ctypes.c_ulonglong * 2)()
    _check(_lib.topo_check_conversions(_ptr(d), _vp(f.data_ptr()), d.numel(),
                                       ctypes.cast(out, _vp)),
           "topo_check_conversions")
    return int(out[0]), int(out[1])


def compliance_noalloc(f, u, c, nrhs=1):
    """c[k] = f_k^T u_k through topo_compliance_noalloc (static library scratch, no allocation).

    f, u: contiguous FP64 CUDA tensors of nrhs * n entries; c: contiguous FP64 CUDA tensor of
    nrhs entries, written asynchronously on the current stream.
    """
    import torch
    if f.numel() != u.numel() or nrhs < 1 or f.numel() % nrhs:
        raise ValueError("f and u must hold nrhs vectors of one length")
    if c.numel() < nrhs:
        raise ValueError("c must hold nrhs entries")
    n = f.numel() // nrhs
    _check(_lib.topo_compliance_noalloc(_ptr(f), _ptr(u), n, int(nrhs), _ptr(c),
                                        _vp(torch.cuda.current_stream().cuda_stream)),
           "topo_compliance_noalloc")
    return c

class IP:
    """Primal-dual interior-point method on the GPU (see include/topo.h)."""

    def __init__(self, nx, ny, nz=0, fixed=None, f=None, V=None, xbar=1.0, levels=3,
                 precision=FP64, nu1=2, nu2=2, omega=None, max_iter=1000, E=1.0, nu=0.3,
                 simp=None, K0=None):
        """simp = (p, rmin): the SIMP model with the density filter (topo_ip_set_simp).
        K0: the caller's element matrix (None: the analytic one from E, nu)."""
        import torch
        d, self._fixed, self.dim, self.n = _desc(nx, ny, nz, fixed, levels, precision, nu1, nu2,
                                                 omega, max_iter, 1, None, E, nu, False, K0=K0)
        self.m = nx * ny * (nz if nz else 1)
        self._f = f
        h = _vp()
        _check(_lib.topo_ip_create(ctypes.byref(d), _ptr(f), float(V), float(xbar),
                                   ctypes.byref(h)), "topo_ip_create")
        self._h = h
        _check(_lib.topo_ip_set_stream(h, _vp(torch.cuda.current_stream().cuda_stream)),
               "topo_ip_set_stream")
        if simp is not None:
            self.set_simp(*simp)

    def set_record_file(self, path):
        """Append one JSON line per linear solve to path (None: stop)."""
        _check(_lib.topo_ip_set_record_file(self._h, None if path is None else str(path).encode()),
               "topo_ip_set_record_file")

    def set_simp(self, p, rmin):
        _check(_lib.topo_ip_set_simp(self._h, float(p), float(rmin)), "topo_ip_set_simp")

    def filtered_density(self):
        """x~ = W x at the current iterate (x without the SIMP model), a device tensor."""
        import torch
        xt = torch.empty(self.m, dtype=torch.float64, device="cuda")
        _check(_lib.topo_ip_filtered_density(self._h, _ptr(xt)), "topo_ip_filtered_density")
        return xt

    def close(self):
        if getattr(self, "_h", None):
            _lib.topo_ip_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, opts):
        _check(_lib.topo_ip_init(self._h, ctypes.byref(opts)), "topo_ip_init")

    def step(self, opts):
        info = IpInfo()
        _check(_lib.topo_ip_step(self._h, ctypes.byref(opts), ctypes.byref(info)), "topo_ip_step")
        return info

    def run(self, opts):
        info = IpInfo()
        _check(_lib.topo_ip_run(self._h, ctypes.byref(opts), ctypes.byref(info)), "topo_ip_run")
        return info

    def set_vcycle_fusion(self, on):
        _check(_lib.topo_ip_set_vcycle_fusion(self._h, int(bool(on))), "topo_ip_set_vcycle_fusion")

    def state(self):
        """(u, x, phi, psi, scal, pw): the iterate, scal = (lambda, s, r, barrier reductions so
        far) on the host, and pw the
        augmented solver's power-iteration vectors with a trailing 1.0 when the next build starts
        from them (0.0: from the fixed start vector)."""
        import torch
        u = torch.empty(self.n, dtype=torch.float64, device="cuda")
        x, phi, psi = (torch.empty(self.m, dtype=torch.float64, device="cuda") for _ in range(3))
        scal = np.zeros(4)
        _check(_lib.topo_ip_get_state(self._h, _ptr(u), _ptr(x), _ptr(phi), _ptr(psi),
                                      scal.ctypes.data_as(_vp)), "topo_ip_get_state")
        ln = ctypes.c_longlong(0)
        _check(_lib.topo_ip_power_state_size(self._h, ctypes.byref(ln)), "topo_ip_power_state_size")
        pw = torch.zeros(ln.value + 1, dtype=torch.float64, device="cuda")
        ready = ctypes.c_int(0)
        _check(_lib.topo_ip_get_power_state(self._h, _ptr(pw), ctypes.byref(ready)),
               "topo_ip_get_power_state")
        pw[ln.value] = float(ready.value)
        return u, x, phi, psi, scal, pw

    def set_state(self, u, x, phi, psi, scal, pw=None):
        scal = np.ascontiguousarray(scal, dtype=np.float64)
        _check(_lib.topo_ip_set_state(self._h, _ptr(u), _ptr(x), _ptr(phi), _ptr(psi),
                                      scal.ctypes.data_as(_vp)), "topo_ip_set_state")
        ln = ctypes.c_longlong(0)
        _check(_lib.topo_ip_power_state_size(self._h, ctypes.byref(ln)), "topo_ip_power_state_size")
        if pw is None:
            _check(_lib.topo_ip_set_power_state(self._h, None, 0), "topo_ip_set_power_state")
            return
        if pw.numel() != ln.value + 1:
            raise ValueError("set_state: power state has %d entries, expected %d"
                             % (pw.numel(), ln.value + 1))
        ready = int(float(pw[ln.value]) != 0.0)
        _check(_lib.topo_ip_set_power_state(self._h, _ptr(pw), ready), "topo_ip_set_power_state")


class OC:
    """OC / DOC / AOC on the GPU (see include/topo.h)."""

    def __init__(self, nx, ny, nz=0, fixed=None, f=None, V=None, xbar=1.0, levels=3,
                 precision=FP64, nu1=2, nu2=2, omega=None, max_iter=1000, E=1.0, nu=0.3,
                 K0=None):
        import torch
        d, self._fixed, self.dim, self.n = _desc(nx, ny, nz, fixed, levels, precision, nu1, nu2,
                                                 omega, max_iter, 1, None, E, nu, False, K0=K0)
        self.m = nx * ny * (nz if nz else 1)
        h = _vp()
        _check(_lib.topo_oc_create(ctypes.byref(d), _ptr(f), float(V), float(xbar),
                                   ctypes.byref(h)), "topo_oc_create")
        self._h = h
        _check(_lib.topo_oc_set_stream(h, _vp(torch.cuda.current_stream().cuda_stream)),
               "topo_oc_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            _lib.topo_oc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_record_file(self, path):
        """Append one JSON line per linear solve to path (None: stop)."""
        _check(_lib.topo_oc_set_record_file(self._h, None if path is None else str(path).encode()),
               "topo_oc_set_record_file")

    def init(self, x0=None):
        _check(_lib.topo_oc_init(self._h, _ptr(x0) if x0 is not None else None), "topo_oc_init")

    def step(self, opts):
        info = OcInfo()
        _check(_lib.topo_oc_step(self._h, ctypes.byref(opts), ctypes.byref(info)), "topo_oc_step")
        return info

    def run(self, opts):
        info = OcInfo()
        _check(_lib.topo_oc_run(self._h, ctypes.byref(opts), ctypes.byref(info)), "topo_oc_run")
        return info

    def x(self):
        import torch
        x = torch.empty(self.m, dtype=torch.float64, device="cuda")
        _check(_lib.topo_oc_get_x(self._h, _ptr(x)), "topo_oc_get_x")
        return x

    def u(self):
        import torch
        u = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(_lib.topo_oc_get_u(self._h, _ptr(u)), "topo_oc_get_u")
        return u

    def state(self):
        """(x, u, scal, pw): the iterate, the warm-start displacement, scal = (CG tolerance,
        previous and last compliance, u-valid flag, linear solves, iterations, CG iterations) on
        the host, and the solver's power-iteration vectors with a trailing ready flag."""
        import torch
        x = torch.empty(self.m, dtype=torch.float64, device="cuda")
        u = torch.empty(self.n, dtype=torch.float64, device="cuda")
        scal = np.zeros(7)
        _check(_lib.topo_oc_get_state(self._h, _ptr(x), _ptr(u), scal.ctypes.data_as(_vp)),
               "topo_oc_get_state")
        ln = ctypes.c_longlong(0)
        _check(_lib.topo_oc_power_state_size(self._h, ctypes.byref(ln)), "topo_oc_power_state_size")
        pw = torch.zeros(ln.value + 1, dtype=torch.float64, device="cuda")
        ready = ctypes.c_int(0)
        _check(_lib.topo_oc_get_power_state(self._h, _ptr(pw), ctypes.byref(ready)),
               "topo_oc_get_power_state")
        pw[ln.value] = float(ready.value)
        return x, u, scal, pw

    def set_state(self, x, u, scal, pw=None):
        scal = np.ascontiguousarray(scal, dtype=np.float64)
        _check(_lib.topo_oc_set_state(self._h, _ptr(x), _ptr(u), scal.ctypes.data_as(_vp)),
               "topo_oc_set_state")
        ln = ctypes.c_longlong(0)
        _check(_lib.topo_oc_power_state_size(self._h, ctypes.byref(ln)), "topo_oc_power_state_size")
        if pw is None:
            _check(_lib.topo_oc_set_power_state(self._h, None, 0), "topo_oc_set_power_state")
            return
        if pw.numel() != ln.value + 1:
            raise ValueError("set_state: power state has %d entries, expected %d"
                             % (pw.numel(), ln.value + 1))
        ready = int(float(pw[ln.value]) != 0.0)
        _check(_lib.topo_oc_set_power_state(self._h, _ptr(pw), ready), "topo_oc_set_power_state")


class Solver:
    """MGCG solver for K(x) u = b on one structured grid (see include/topo.h)."""

    def __init__(self, nx, ny, nz=0, fixed=None, levels=3, precision=FP64, nu1=2, nu2=2,
                 omega=None, max_iter=1000, nrhs=1, flexible=None, E=1.0, nu=0.3,
                 generic_kernels=False, omega_auto=False, smoother=0, K0=None):
        dim = 3 if nz else 2
        n = dim * (nx + 1) * (ny + 1) * ((nz + 1) if nz else 1)
        if fixed is None:
            fixed = np.zeros(n, dtype=np.uint8)
        self._fixed = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
        if self._fixed.size != n:
            raise ValueError("fixed mask has %d entries, expected %d" % (self._fixed.size, n))
        if omega is None:
            omega = 0.6 if dim == 2 else 0.5
        if flexible is None:
            flexible = 0
        k0 = _k0_array(dim, K0)
        d = SolverDesc(dim, nx, ny, nz, E, nu,
                       self._fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), levels,
                       precision, nu1, nu2, omega, max_iter, nrhs, flexible, int(generic_kernels),
                       int(smoother), int(omega_auto),
                       None if k0 is None else k0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        h = _vp()
        _check(_lib.topo_solver_create(ctypes.byref(d), ctypes.byref(h)), "topo_solver_create")
        self._h = h
        self.dim, self.nx, self.ny, self.nz = dim, nx, ny, nz
        self.n, self.m = n, nx * ny * (nz if nz else 1)
        self.levels, self.precision, self.nrhs = levels, precision, nrhs
        import torch
        _check(_lib.topo_set_stream(self._h, _vp(torch.cuda.current_stream().cuda_stream)),
               "topo_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            _lib.topo_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_wait_limit_ns(self, ns):
        """Bound of the device-side waits (topo_set_wait_limit_ns; 0: expire at once)."""
        _check(_lib.topo_set_wait_limit_ns(self._h, int(ns)), "topo_set_wait_limit_ns")

    def set_sweep_rows(self, rows):
        """Strip height of the 2D finest-level FP32 sweeps (topo_set_sweep_rows; 0: automatic)."""
        _check(_lib.topo_set_sweep_rows(self._h, int(rows)), "topo_set_sweep_rows")

    def set_record_file(self, path):
        """Append one JSON line per solve to path (topo_set_record_file; None: stop)."""
        _check(_lib.topo_set_record_file(self._h, None if path is None else str(path).encode()),
               "topo_set_record_file")

    @property
    def device_bytes(self):
        return int(_lib.topo_solver_device_bytes(self._h))

    @property
    def launch_count(self):
        return int(_lib.topo_solver_launch_count(self._h))

    def set_graph_mode(self, mode):
        """0: replayed graph of 4 CG iterations (default); 1: one conditional-while graph per solve."""
        _check(_lib.topo_set_graph_mode(self._h, int(mode)), "topo_set_graph_mode")

    def set_profiling(self, on):
        _check(_lib.topo_set_profiling(self._h, int(bool(on))), "topo_set_profiling")

    def set_outer_precision(self, mode):
        """Outer CG operator on the 2D finest level: 0 FP64, 1 float pairs (mixed default)."""
        _check(_lib.topo_set_outer_precision(self._h, int(mode)), "topo_set_outer_precision")

    def set_vcycle_fusion(self, on):
        """Fuse the deep levels of the 2D V-cycle into one cluster launch (default on)."""
        _check(_lib.topo_set_vcycle_fusion(self._h, int(bool(on))), "topo_set_vcycle_fusion")

    def set_profiling_mask(self, mask):
        """Profile the kinds in mask (bit k = PROFILE_KINDS[k]); 0 turns profiling off."""
        _check(_lib.topo_set_profiling_mask(self._h, int(mask)), "topo_set_profiling_mask")

    def profile(self):
        """(summed ms, launches) of the outer operator kernel since set_profiling."""
        ms, cnt = ctypes.c_double(), ctypes.c_longlong()
        _check(_lib.topo_get_profile(self._h, ctypes.byref(ms), ctypes.byref(cnt)), "topo_get_profile")
        return ms.value, cnt.value

    PROFILE_KINDS = ("outer_operator", "fine_smoothing_sweep", "fine_residual",
                     "fine_restriction", "fine_prolongation", "vcycle", "vcycle_levels_ge1",
                     "vcycle_levels_ge2", "vcycle_levels_ge3", "vcycle_levels_ge4",
                     "vcycle_levels_ge5", "vcycle_levels_ge6")

    def profile_kernel(self, kind):
        """(summed ms, launches) of one profiled kernel kind (index into PROFILE_KINDS)."""
        ms, cnt = ctypes.c_double(), ctypes.c_longlong()
        _check(_lib.topo_get_profile_kernel(self._h, int(kind), ctypes.byref(ms), ctypes.byref(cnt)),
               "topo_get_profile_kernel")
        return ms.value, cnt.value

    def set_density(self, x):
        _check(_lib.topo_set_density(self._h, _ptr(x)), "topo_set_density")

    def solve(self, b, u=None, tol=1e-8, use_x0=False, allow_not_converged=False):
        import torch
        if u is None:
            u = torch.zeros_like(b)
        info = SolveInfo()
        allow = (E_NOT_CONVERGED,) if allow_not_converged else ()
        _check(_lib.topo_solve(self._h, _ptr(b), _ptr(u), float(tol), int(bool(use_x0)),
                               ctypes.byref(info)), "topo_solve", allow)
        return u, info

    def solve_host(self, x, b, u, tol=1e-8, allow_not_converged=False):
        """topo_solve_host: densities x, right-hand sides b and the solution u in host memory
        (contiguous FP64 CPU tensors, best page-locked)."""
        for t in (x, b, u):
            if t.is_cuda or t.dtype != _torch_f64() or not t.is_contiguous():
                raise ValueError("expected contiguous float64 CPU tensors")
        info = SolveInfo()
        allow = (E_NOT_CONVERGED,) if allow_not_converged else ()
        _check(_lib.topo_solve_host(self._h, _vp(x.data_ptr()), _vp(b.data_ptr()),
                                    _vp(u.data_ptr()), float(tol), ctypes.byref(info)),
               "topo_solve_host", allow)
        return info

    def apply_K(self, v, y=None):
        import torch
        y = torch.empty_like(v) if y is None else y
        _check(_lib.topo_apply_K(self._h, _ptr(v), _ptr(y)), "topo_apply_K")
        return y

    def apply_vcycle(self, r, y=None):
        import torch
        y = torch.empty_like(r) if y is None else y
        _check(_lib.topo_apply_vcycle(self._h, _ptr(r), _ptr(y)), "topo_apply_vcycle")
        return y

    def level_matrices(self, level):
        m = _lib.topo_level_elems(self._h, level)
        ne = 8 if self.dim == 2 else 24
        out = np.zeros((m, ne, ne))
        _check(_lib.topo_get_level_matrices(self._h, level, out.ctypes.data_as(_vp)),
               "topo_get_level_matrices")
        return out

    def compliance(self, f, u):
        c = np.zeros(self.nrhs)
        _check(_lib.topo_compliance(self._h, _ptr(f), _ptr(u), c.ctypes.data_as(_vp)),
               "topo_compliance")
        return c

    def element_energy(self, u, out=None):
        import torch
        out = torch.empty(self.m, dtype=torch.float64, device=u.device) if out is None else out
        _check(_lib.topo_element_energy(self._h, _ptr(u), _ptr(out)), "topo_element_energy")
        return out

    def grad_x(self, lam, u, out=None):
        import torch
        out = torch.empty(self.m, dtype=torch.float64, device=u.device) if out is None else out
        _check(_lib.topo_grad_x(self._h, _ptr(lam), _ptr(u), _ptr(out)), "topo_grad_x")
        return out


def exported_symbols():
    """Names of the C-ABI entry points this binding expects (for the symbol check)."""
    return sorted(_SIGS)
