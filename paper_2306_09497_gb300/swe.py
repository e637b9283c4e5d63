"""Thin ctypes binding of ``libswe_gb300.so`` (C ABI in ``include/swe_gb300.h``).

Argument marshalling only: every computation runs in the CUDA library.  Device
arrays are passed as torch tensors (their data pointers) or raw integer
addresses; streams default to torch's current CUDA stream.  There is no CPU
fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

from .build import lib_path

SWE_OK, SWE_EINVAL, SWE_ENOMEM, SWE_ECUDA, SWE_EUNSTABLE, SWE_ETIMEOUT, SWE_ENOTCONV = range(7)
SWE_FP64, SWE_SPLIT_BF16X3 = 0, 1
SWE_IMEX, SWE_SLSI_SETTLS, SWE_SLSI_SETTLS_1STEP = 0, 1, 2

STATUS_NAMES = {0: "SWE_OK", 1: "SWE_EINVAL", 2: "SWE_ENOMEM", 3: "SWE_ECUDA", 4: "SWE_EUNSTABLE",
                5: "SWE_ETIMEOUT", 6: "SWE_ENOTCONV"}

# Every symbol include/swe_gb300.h declares (checked by the CPU test suite).
EXPORTED = [
    "swe_version", "swe_last_error", "swe_ncoef", "swe_plan_create", "swe_plan_destroy", "swe_plan_gauss",
    "sht_inverse", "sht_forward", "swe_nonlinear", "swe_linear", "swe_implicit_solve", "swe_balance",
    "propagate_F", "propagate_G", "swe_pint_create", "swe_pint_destroy", "swe_pint_init", "parareal_iterate",
    "swe_pint_solution", "swe_pint_load", "swe_pint_save", "swe_launch_count", "swe_prof_enable",
    "swe_prof_reset", "swe_prof_read", "sht_inverse_noalloc", "swe_mgrit_create", "swe_mgrit_destroy",
    "swe_mgrit_init", "mgrit_cycle", "swe_mgrit_cpoints", "swe_server_create", "swe_server_destroy",
    "swe_server_submit", "swe_server_step", "swe_server_result", "swe_server_norms", "swe_plan_check",
    "swe_plan_inject_status", "swe_wait_selftest", "swe_error_norms", "swe_ke_spectrum", "swe_stability_region",
    "swe_request_bytes", "swe_plan_set_nphi_form", "swe_plan_set_legendre_mode", "swe_plan_tuning",
]
SWE_NPHI_FLUX, SWE_NPHI_ADVECTIVE = 0, 1
SWE_LEGENDRE_AUTO, SWE_LEGENDRE_PERSISTENT, SWE_LEGENDRE_PER_TILE = 0, 1, 2
SWE_STAB_COARSE_ALONE, SWE_STAB_PARAREAL, SWE_STAB_MGRIT2, SWE_STAB_MGRIT2_PRINTED = range(4)
SWE_METHOD_PARAREAL, SWE_METHOD_MGRIT2 = 0, 1


class SWEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ct.Structure):
    _fields_ = [("M", ct.c_int), ("nlat", ct.c_int), ("nlon", ct.c_int), ("a", ct.c_double),
                ("omega", ct.c_double), ("g", ct.c_double), ("phibar", ct.c_double), ("prec", ct.c_int)]


class StepperDesc(ct.Structure):
    _fields_ = [("scheme", ct.c_int), ("dt", ct.c_double), ("nsteps", ct.c_int), ("visc_q", ct.c_int),
                ("visc_nu", ct.c_double)]


class PintDesc(ct.Structure):
    _fields_ = [("fine_plan", ct.c_void_p), ("coarse_plan", ct.c_void_p), ("fine", StepperDesc),
                ("coarse", StepperDesc), ("S", ct.c_int), ("use_graphs", ct.c_int)]


class MgritDesc(ct.Structure):
    _fields_ = [("L", ct.c_int), ("cf", ct.c_int), ("nu", ct.c_int), ("N0", ct.c_int), ("cycle", ct.c_int),
                ("plan", ct.c_void_p * 8), ("step", StepperDesc * 8)]


class StabilityDesc(ct.Structure):
    _fields_ = [("coarse_scheme", ct.c_int), ("method", ct.c_int), ("n", ct.c_int), ("k", ct.c_int),
                ("cf", ct.c_int), ("Nc", ct.c_int), ("nu", ct.c_int), ("n_kappa", ct.c_int),
                ("xiL_re", ct.c_double), ("xiL_im", ct.c_double)]


class ServerDesc(ct.Structure):
    _fields_ = [("hbm_budget_bytes", ct.c_size_t), ("max_active", ct.c_int)]


class RequestDesc(ct.Structure):
    _fields_ = [("fine_plan", ct.c_void_p), ("coarse_plan", ct.c_void_p), ("method", ct.c_int),
                ("fine", StepperDesc), ("coarse", StepperDesc), ("S", ct.c_int), ("cf", ct.c_int),
                ("nu_relax", ct.c_int), ("iters", ct.c_int), ("U0_host", ct.c_void_p)]


_lib = None


def load(path: Optional[str] = None) -> ct.CDLL:
    """Load the CUDA library (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ct.CDLL(path)
    vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
    sigs = {
        "swe_version": ([], ct.c_char_p),
        "swe_last_error": ([], ct.c_char_p),
        "swe_ncoef": ([i], ct.c_int64),
        "swe_plan_create": ([ct.POINTER(PlanDesc), ct.POINTER(vp)], i),
        "swe_plan_destroy": ([vp], i),
        "swe_plan_gauss": ([vp, vp, vp], i),
        "sht_inverse": ([vp, vp, vp, i, vp], i),
        "sht_forward": ([vp, vp, vp, i, vp], i),
        "swe_nonlinear": ([vp, vp, vp, i, vp], i),
        "swe_linear": ([vp, vp, vp, i, vp], i),
        "swe_implicit_solve": ([vp, d, vp, vp, i, vp], i),
        "swe_balance": ([vp, vp, vp, vp, i, vp], i),
        "propagate_F": ([vp, ct.POINTER(StepperDesc), vp, vp, i, vp], i),
        "propagate_G": ([vp, vp, ct.POINTER(StepperDesc), vp, vp, i, vp], i),
        "swe_pint_create": ([ct.POINTER(PintDesc), ct.POINTER(vp)], i),
        "swe_pint_destroy": ([vp], i),
        "swe_pint_init": ([vp, vp, vp], i),
        "parareal_iterate": ([vp, i, d, ct.POINTER(i), ct.POINTER(d), vp], i),
        "swe_pint_solution": ([vp, vp, vp], i),
        "swe_pint_load": ([vp, vp, vp, vp], i),
        "swe_pint_save": ([vp, vp, vp, vp], i),
        "swe_launch_count": ([], ct.c_longlong),
        "swe_prof_enable": ([i], i),
        "swe_prof_reset": ([], None),
        "swe_prof_read": ([i, ct.c_char_p, i, ct.POINTER(ct.c_longlong), ct.POINTER(d), ct.POINTER(d),
                           ct.POINTER(d)], i),
        "sht_inverse_noalloc": ([vp, vp, vp, i, vp], i),
        "swe_mgrit_create": ([ct.POINTER(MgritDesc), ct.POINTER(vp)], i),
        "swe_mgrit_destroy": ([vp], i),
        "swe_mgrit_init": ([vp, vp, vp], i),
        "mgrit_cycle": ([vp, i, d, ct.POINTER(i), ct.POINTER(d), vp], i),
        "swe_mgrit_cpoints": ([vp, vp, vp], i),
        "swe_server_create": ([ct.POINTER(ServerDesc), ct.POINTER(vp)], i),
        "swe_server_destroy": ([vp], i),
        "swe_server_submit": ([vp, ct.POINTER(RequestDesc), ct.POINTER(ct.c_longlong)], i),
        "swe_server_step": ([vp, ct.POINTER(i), ct.POINTER(i), ct.POINTER(i)], i),
        "swe_server_result": ([vp, ct.c_longlong, vp, vp], i),
        "swe_server_norms": ([vp, ct.c_longlong, vp, i, ct.POINTER(i)], i),
        "swe_plan_check": ([vp, vp], i),
        "swe_plan_inject_status": ([vp, i, vp], i),
        "swe_wait_selftest": ([vp, ct.c_longlong, vp], i),
        "swe_error_norms": ([vp, vp, vp, i, i, vp, vp], i),
        "swe_ke_spectrum": ([vp, vp, i, vp, vp], i),
        "swe_stability_region": ([ct.POINTER(StabilityDesc), d, d, i, d, d, i, vp, vp], i),
        "swe_request_bytes": ([ct.POINTER(RequestDesc), ct.POINTER(ct.c_size_t)], i),
        "swe_plan_set_nphi_form": ([vp, i], i),
        "swe_plan_set_legendre_mode": ([vp, i], i),
        "swe_plan_tuning": ([vp, ct.c_char_p, ct.c_size_t], i),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int):
    if status != SWE_OK:
        raise SWEError(status, load().swe_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def ncoef(M: int) -> int:
    return int(load().swe_ncoef(M))


def stepper(scheme=SWE_IMEX, dt=60.0, nsteps=1, visc_q=2, visc_nu=0.0) -> StepperDesc:
    return StepperDesc(scheme, dt, nsteps, visc_q, visc_nu)


class Plan:
    """A truncation T_M on an nlat x nlon Gaussian grid (swe_plan_create)."""

    def __init__(self, M, nlat, nlon, a=6371.22e3, omega=7.292e-5, g=9.80616, phibar=1.0e5, prec=SWE_FP64):
        lib = load()
        self.M, self.nlat, self.nlon, self.prec = M, nlat, nlon, prec
        self.a, self.omega, self.g, self.phibar = a, omega, g, phibar
        desc = PlanDesc(M, nlat, nlon, a, omega, g, phibar, prec)
        h = ct.c_void_p()
        _check(lib.swe_plan_create(ct.byref(desc), ct.byref(h)))
        self.h = h
        self.nc = ncoef(M)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().swe_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_nphi_form(self, form):
        """SWE_NPHI_FLUX (default) or SWE_NPHI_ADVECTIVE geopotential tendency (see the C header)."""
        _check(load().swe_plan_set_nphi_form(self.h, form))

    def set_legendre_mode(self, mode):
        """SWE_LEGENDRE_AUTO (default), _PERSISTENT or _PER_TILE tensor-core Legendre kernels."""
        _check(load().swe_plan_set_legendre_mode(self.h, mode))

    def tuning(self) -> str:
        """Launch configurations chosen so far (ring kernel, Legendre variants with their times)."""
        buf = ct.create_string_buffer(4096)
        _check(load().swe_plan_tuning(self.h, buf, len(buf)))
        return buf.value.decode()

    def check(self, stream=None):
        """Synchronise the stream and return the plan's status (SWE_OK, SWE_ETIMEOUT or
        SWE_EUNSTABLE); the status word is cleared.  Does not raise."""
        return int(load().swe_plan_check(self.h, _stream(stream)))

    def inject_status(self, bits, stream=None):
        """Host-side fault injection into the status word (1 non-finite, 2 timeout)."""
        _check(load().swe_plan_inject_status(self.h, bits, _stream(stream)))

    def wait_selftest(self, polls, stream=None):
        """Bounded-wait diagnostic: a wait that nothing completes gives up after `polls` polls."""
        _check(load().swe_wait_selftest(self.h, polls, _stream(stream)))

    def error_norms(self, U, Uref, S, R_norm, stream=None):
        """[S][3][2] numpy array: (E_{psi,R} of Eq. 21, area-weighted relative L2) per state and field."""
        import numpy as np
        out = np.empty((S, 3, 2), dtype=np.float64)
        _check(load().swe_error_norms(self.h, _ptr(U), _ptr(Uref), S, R_norm, out.ctypes.data, _stream(stream)))
        return out

    def ke_spectrum(self, U, S, E, stream=None):
        """KE spectrum E[s][n], n = 0..M, into the device array E ([S][M+1] float64)."""
        _check(load().swe_ke_spectrum(self.h, _ptr(U), S, _ptr(E), _stream(stream)))

    def gauss(self):
        import numpy as np
        mu = np.empty(self.nlat)
        w = np.empty(self.nlat)
        _check(load().swe_plan_gauss(self.h, mu.ctypes.data, w.ctypes.data))
        return mu, w

    # -- transforms --------------------------------------------------------
    def sht_inverse(self, spec, grid, batch, stream=None):
        _check(load().sht_inverse(self.h, _ptr(spec), _ptr(grid), batch, _stream(stream)))

    def sht_inverse_noalloc(self, spec, grid, batch, stream=None):
        """sht_inverse without any device allocation (static 64 MiB scratch; see the C header)."""
        _check(load().sht_inverse_noalloc(self.h, _ptr(spec), _ptr(grid), batch, _stream(stream)))

    def sht_forward(self, grid, spec, batch, stream=None):
        _check(load().sht_forward(self.h, _ptr(grid), _ptr(spec), batch, _stream(stream)))

    # -- operators ---------------------------------------------------------
    def nonlinear(self, U, N, S, stream=None):
        _check(load().swe_nonlinear(self.h, _ptr(U), _ptr(N), S, _stream(stream)))

    def linear(self, U, LU, S, stream=None):
        _check(load().swe_linear(self.h, _ptr(U), _ptr(LU), S, _stream(stream)))

    def implicit_solve(self, alpha, R, X, S, stream=None):
        _check(load().swe_implicit_solve(self.h, alpha, _ptr(R), _ptr(X), S, _stream(stream)))

    def balance(self, xi, phi_add, U, S, stream=None):
        _check(load().swe_balance(self.h, _ptr(xi), _ptr(phi_add), _ptr(U), S, _stream(stream)))

    def propagate(self, st: StepperDesc, U_in, U_out, S, stream=None):
        _check(load().propagate_F(self.h, ct.byref(st), _ptr(U_in), _ptr(U_out), S, _stream(stream)))

    def propagate_G(self, fine: Optional["Plan"], st: StepperDesc, U_in, U_out, S, stream=None):
        fh = fine.h if fine is not None else None
        _check(load().propagate_G(self.h, fh, ct.byref(st), _ptr(U_in), _ptr(U_out), S, _stream(stream)))


class Parareal:
    """Parareal on S slices (swe_pint_create / swe_pint_init / parareal_iterate)."""

    def __init__(self, fine_plan: Plan, coarse_plan: Plan, fine: StepperDesc, coarse: StepperDesc, S: int,
                 use_graphs: bool = True):
        lib = load()
        self.fine_plan, self.coarse_plan, self.S = fine_plan, coarse_plan, S
        desc = PintDesc(fine_plan.h, coarse_plan.h, fine, coarse, S, 1 if use_graphs else 0)
        h = ct.c_void_p()
        _check(lib.swe_pint_create(ct.byref(desc), ct.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().swe_pint_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, U0, stream=None):
        _check(load().swe_pint_init(self.h, _ptr(U0), _stream(stream)))

    def iterate(self, kmax: int, tol: float = 0.0, stream=None):
        """Returns (iterations run, list of per-iteration convergence norms)."""
        k = ct.c_int(0)
        hist = (ct.c_double * max(kmax, 1))()
        st = load().parareal_iterate(self.h, kmax, tol, ct.byref(k), hist, _stream(stream))
        norms = [hist[i] for i in range(k.value)]
        _check(st)
        return k.value, norms

    def solution(self, U_out, stream=None):
        _check(load().swe_pint_solution(self.h, _ptr(U_out), _stream(stream)))

    def load_state(self, U, Gold=None, stream=None):
        """Resume from (U^k_n, phi_c(U^k_n)); host or device arrays."""
        _check(load().swe_pint_load(self.h, _ptr(U), _ptr(Gold), _stream(stream)))

    def save_state(self, U, Gold=None, stream=None):
        """Checkpoint (U^k_n, phi_c(U^k_n)) into host or device arrays."""
        _check(load().swe_pint_save(self.h, _ptr(U), _ptr(Gold), _stream(stream)))


class MGRIT:
    """MGRIT over L levels (swe_mgrit_create / swe_mgrit_init / mgrit_cycle)."""

    def __init__(self, plans, steps, N0: int, cf: int, nu: int = 0, cycle: int = 1):
        L = len(plans)
        assert len(steps) == L and 2 <= L <= 8
        desc = MgritDesc()
        desc.L, desc.cf, desc.nu, desc.N0, desc.cycle = L, cf, nu, N0, cycle
        for l in range(L):
            desc.plan[l] = plans[l].h.value
            desc.step[l] = steps[l]
        self.plans, self.N0, self.cf = plans, N0, cf
        h = ct.c_void_p()
        _check(load().swe_mgrit_create(ct.byref(desc), ct.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().swe_mgrit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, U0, stream=None):
        _check(load().swe_mgrit_init(self.h, _ptr(U0), _stream(stream)))

    def cycle(self, ncycles: int, tol: float = 0.0, stream=None):
        k = ct.c_int(0)
        hist = (ct.c_double * max(ncycles, 1))()
        st = load().mgrit_cycle(self.h, ncycles, tol, ct.byref(k), hist, _stream(stream))
        norms = [hist[i] for i in range(k.value)]
        _check(st)
        return k.value, norms

    def cpoints(self, U_out, stream=None):
        _check(load().swe_mgrit_cpoints(self.h, _ptr(U_out), _stream(stream)))


class Server:
    """Continuous-batching forecast server (swe_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int):
        h = ct.c_void_p()
        _check(load().swe_server_create(ct.byref(ServerDesc(hbm_budget_bytes, max_active)), ct.byref(h)))
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().swe_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, fine_plan: Plan, coarse_plan: Plan, method: int, fine: StepperDesc, coarse: StepperDesc,
               S: int, iters: int, U0_host, cf: int = 1, nu_relax: int = 0) -> int:
        """U0_host: numpy complex128 [3][NC] (copied)."""
        import numpy as np
        u0 = np.ascontiguousarray(U0_host, dtype=np.complex128)
        d = RequestDesc(fine_plan.h.value, coarse_plan.h.value, method, fine, coarse, S, cf, nu_relax, iters,
                        u0.ctypes.data)
        rid = ct.c_longlong(0)
        _check(load().swe_server_submit(self.h, ct.byref(d), ct.byref(rid)))
        self._keep[rid.value] = (S, fine_plan.nc)
        return rid.value

    @staticmethod
    def request_bytes(fine_plan: Plan, coarse_plan: Plan, method: int, fine: StepperDesc, coarse: StepperDesc,
                      S: int, iters: int = 1, U0_host=None, cf: int = 1, nu_relax: int = 0) -> int:
        """Device memory the server charges to such a request (swe_request_bytes)."""
        d = RequestDesc(fine_plan.h.value, coarse_plan.h.value, method, fine, coarse, S, cf, nu_relax, iters, None)
        n = ct.c_size_t(0)
        _check(load().swe_request_bytes(ct.byref(d), ct.byref(n)))
        return n.value

    def step(self):
        a, q, dn = ct.c_int(0), ct.c_int(0), ct.c_int(0)
        _check(load().swe_server_step(self.h, ct.byref(a), ct.byref(q), ct.byref(dn)))
        return a.value, q.value, dn.value

    def result(self, rid: int):
        """(states [S+1][3][NC] complex128, latency s, queueing s, iterations) of a finished request."""
        import numpy as np
        S, nc = self._keep[rid]
        out = np.empty((S + 1, 3, nc), dtype=np.complex128)
        tm = (ct.c_double * 3)()
        _check(load().swe_server_result(self.h, rid, out.ctypes.data, tm))
        del self._keep[rid]
        return out, tm[0], tm[1], int(tm[2])

    def norms(self, rid: int):
        buf = (ct.c_double * 64)()
        n = ct.c_int(0)
        _check(load().swe_server_norms(self.h, rid, buf, 64, ct.byref(n)))
        return [buf[i] for i in range(min(n.value, 64))]


def stability_region(out, coarse_scheme, method, xiL, re, im, n=100, k=0, cf=2, Nc=1, nu=0, n_kappa=21,
                     stream=None):
    """|A| over the xi_N grid re = (re0, re1, nre) x im = (im0, im1, nim) into the device array
    out [nim][nre] (float64); see swe_stability_region in the C header."""
    xiL = complex(xiL)
    desc = StabilityDesc(coarse_scheme, method, n, k, cf, Nc, nu, n_kappa, xiL.real, xiL.imag)
    _check(load().swe_stability_region(ct.byref(desc), re[0], re[1], re[2], im[0], im[1], im[2], _ptr(out),
                                       _stream(stream)))


def launch_count() -> int:
    return int(load().swe_launch_count())


def prof_enable(on: bool) -> bool:
    return bool(load().swe_prof_enable(1 if on else 0))


def prof_reset():
    load().swe_prof_reset()


def prof_stats():
    """{kernel name: (timed launches, total ms, algorithmic flops, algorithmic bytes)}."""
    lib = load()
    out = {}
    i = 0
    name = ct.create_string_buffer(64)
    while True:
        n, ms, fl, by = ct.c_longlong(), ct.c_double(), ct.c_double(), ct.c_double()
        if not lib.swe_prof_read(i, name, 64, ct.byref(n), ct.byref(ms), ct.byref(fl), ct.byref(by)):
            break
        out[name.value.decode()] = (n.value, ms.value, fl.value, by.value)
        i += 1
    return out
