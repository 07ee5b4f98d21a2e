"""Thin ctypes binding of the libpyro C ABI (``include/pyro.h``).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Arrays may be torch CUDA tensors (device pointers, launched on
torch's current stream) or numpy arrays (host pointers, staged by the library).
All arrays are float64, contiguous, species-major: ``Y[k, p]``.

There is no CPU fallback: if ``libpyro.so`` cannot be loaded the import of
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libpyro.so")

PYRO_OK = 0
PYRO_EINVAL = -1
PYRO_ECUDA = -2
PYRO_ECOMPILE = -3
PYRO_EMECH = -4
PYRO_ENOCONV = -5
PYRO_ENOMLP = -6

# every entry point declared in include/pyro.h
EXPORTS = [
    "pyro_mech_load", "pyro_mech_free", "pyro_mech_info", "pyro_mech_stat", "pyro_mech_source",
    "pyro_density", "pyro_internal_energy", "pyro_temperature", "pyro_net_production_rates",
    "pyro_nonconverged", "pyro_math_eval", "pyro_last_error", "pyro_version",
    "pyro_net_production_rates_noalloc", "pyro_mech_prepare", "pyro_jvp", "pyro_vjp", "pyro_jacobian",
    "pyro_mlp_n_params", "pyro_mlp_set_params", "pyro_mlp_get_params", "pyro_mlp_train", "pyro_mlp_grad",
    "pyro_mlp_guess", "pyro_mlp_save", "pyro_mlp_load", "pyro_enthalpy", "pyro_temperature_enthalpy",
    "pyro_jacobian_adiabatic", "pyro_cn_step", "pyro_transport",
]

_lib = None


class PyroError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libpyro error %d: %s" % (code, msg))
        self.code = code


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpyro.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2503_24286_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        L.pyro_mech_load.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
        L.pyro_mech_free.argtypes = [P]
        L.pyro_mech_free.restype = None
        L.pyro_mech_info.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
        L.pyro_mech_stat.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
        L.pyro_mech_source.argtypes = [P]
        L.pyro_mech_source.restype = ctypes.c_char_p
        L.pyro_density.argtypes = [P, I64, D, D, D, D, P]
        L.pyro_internal_energy.argtypes = [P, I64, D, D, D, D, P]
        L.pyro_temperature.argtypes = [P, I64, D, D, D, ctypes.c_int, D, D, P]
        L.pyro_enthalpy.argtypes = [P, I64, D, D, D, D, P]
        L.pyro_jacobian_adiabatic.argtypes = [P, I64, D, D, D, D, P]
        L.pyro_transport.argtypes = [P, I64, D, D, D, D, D, P]
        L.pyro_cn_step.argtypes = [P, I64, ctypes.c_double, D, D, D, ctypes.c_double, ctypes.c_int, D, D, D, P]
        L.pyro_temperature_enthalpy.argtypes = [P, I64, D, D, D, D, D, P]
        L.pyro_net_production_rates.argtypes = [P, I64, D, D, ctypes.c_int, D, D, D, P]
        L.pyro_net_production_rates_noalloc.argtypes = [P, I64, D, D, ctypes.c_int, D, D, D, P]
        L.pyro_mech_prepare.argtypes = [P, ctypes.c_char_p]
        L.pyro_jvp.argtypes = [P, I64, D, D, D, D, D, D, D, P]
        L.pyro_vjp.argtypes = [P, I64, D, D, D, D, D, D, D, P]
        L.pyro_jacobian.argtypes = [P, I64, D, D, D, D, P]
        L.pyro_mlp_n_params.argtypes = [P]
        L.pyro_mlp_set_params.argtypes = [P, D, D]
        L.pyro_mlp_get_params.argtypes = [P, D, D]
        L.pyro_mlp_train.argtypes = [P, I64, D, D, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), P]
        L.pyro_mlp_grad.argtypes = [P, I64, D, D, D, ctypes.POINTER(ctypes.c_double), D]
        L.pyro_mlp_guess.argtypes = [P, I64, D, D, D, D, P]
        L.pyro_mlp_save.argtypes = [P, ctypes.c_char_p]
        L.pyro_mlp_load.argtypes = [P, ctypes.c_char_p]
        L.pyro_nonconverged.argtypes = [P, P, ctypes.POINTER(ctypes.c_int64)]
        L.pyro_math_eval.argtypes = [P, ctypes.c_int, I64, D, D, P]
        L.pyro_last_error.restype = ctypes.c_char_p
        L.pyro_last_error.argtypes = []
        L.pyro_version.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != PYRO_OK:
        raise PyroError(rc, lib().pyro_last_error().decode())


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, is_device) of a float64/int32 contiguous array or None."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a.is_cuda
    if not a.flags.c_contiguous:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), False


def _stream(arrays):
    dev = [a for a in arrays if a is not None and _is_torch(a) and a.is_cuda]
    if dev:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(dev[0].device).cuda_stream)
    return ctypes.c_void_p(0)


def _empty_like(ref, shape, dtype="float64"):
    if _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=getattr(torch, dtype), device=ref.device)
    return np.empty(shape, dtype=dtype)


def _n(a) -> int:
    return int(a.shape[-1])


class Mechanism:
    """A loaded, compiled mechanism (``pyro_mech_load``)."""

    def __init__(self, path: str, options: Optional[str] = None):
        L = lib()
        h = ctypes.c_void_p()
        _check(L.pyro_mech_load(path.encode(), options.encode() if options else None, ctypes.byref(h)))
        self._h = h
        ns, nr = ctypes.c_int(), ctypes.c_int()
        W = ctypes.POINTER(ctypes.c_double)()
        _check(L.pyro_mech_info(h, ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(W)))
        self.n_species, self.n_reactions = ns.value, nr.value
        self.W = np.array([W[i] for i in range(ns.value)])

    def close(self):
        if getattr(self, "_h", None):
            lib().pyro_mech_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def stat(self, key: str) -> float:
        v = ctypes.c_double()
        _check(lib().pyro_mech_stat(self._h, key.encode(), ctypes.byref(v)))
        return v.value

    def source(self) -> str:
        return lib().pyro_mech_source(self._h).decode()

    # --- entry points ---------------------------------------------------------
    def density(self, p, T, Y, out=None):
        out = _empty_like(T, (_n(T),)) if out is None else out
        args = [p, T, Y, out]
        _check(lib().pyro_density(self._h, _n(T), *[_ptr(a)[0] for a in args], _stream(args)))
        return out

    def internal_energy(self, T, Y, with_cv=False):
        e = _empty_like(T, (_n(T),))
        cv = _empty_like(T, (_n(T),)) if with_cv else None
        args = [T, Y, e, cv]
        _check(lib().pyro_internal_energy(self._h, _n(T), *[_ptr(a)[0] for a in args], _stream(args)))
        return (e, cv) if with_cv else e

    def enthalpy(self, T, Y, with_cp=False):
        h = _empty_like(T, (_n(T),))
        cp = _empty_like(T, (_n(T),)) if with_cp else None
        args = [T, Y, h, cp]
        _check(lib().pyro_enthalpy(self._h, _n(T), *[_ptr(a)[0] for a in args], _stream(args)))
        return (h, cp) if with_cp else h

    def temperature_enthalpy(self, h, Y, guess=None, with_iters=False, out=None):
        T = _empty_like(h, (_n(h),)) if out is None else out
        it = _empty_like(h, (_n(h),), "int32") if with_iters else None
        args = [h, Y, guess, T, it]
        _check(lib().pyro_temperature_enthalpy(self._h, _n(h), *[_ptr(a)[0] for a in args], _stream(args)))
        return (T, it) if with_iters else T

    def temperature(self, e, Y, guess=None, learned=False, with_iters=False, out=None):
        T = _empty_like(e, (_n(e),)) if out is None else out
        it = _empty_like(e, (_n(e),), "int32") if with_iters else None
        args = [e, Y, guess, T, it]
        ptrs = [_ptr(a)[0] for a in args]
        _check(lib().pyro_temperature(self._h, _n(e), ptrs[0], ptrs[1], ptrs[2], 1 if learned else 0,
                                      ptrs[3], ptrs[4], _stream(args)))
        return (T, it) if with_iters else T

    def net_production_rates(self, rho, Y, T=None, e=None, T_out=None, out=None):
        """omega [N, n] from (rho, T, Y), or from (rho, e, Y) with T solved (returns (omega, T))."""
        if (T is None) == (e is None):
            raise ValueError("give exactly one of T or e")
        n = _n(rho)
        w = _empty_like(rho, (self.n_species, n)) if out is None else out
        energy = e is not None
        if energy and T_out is None:
            T_out = _empty_like(rho, (n,))
        args = [rho, e if energy else T, Y, T_out if energy else None, w]
        ptrs = [_ptr(a)[0] for a in args]
        _check(lib().pyro_net_production_rates(self._h, n, ptrs[0], ptrs[1], 1 if energy else 0, ptrs[2],
                                               ptrs[3], ptrs[4], _stream(args)))
        return (w, T_out) if energy else w

    def net_production_rates_noalloc(self, rho, Y, T=None, e=None, T_out=None, out=None):
        """As :meth:`net_production_rates`, through the entry point that allocates no
        device memory (fixed scratch; synchronous; bounded number of states per call)."""
        if (T is None) == (e is None):
            raise ValueError("give exactly one of T or e")
        n = _n(rho)
        w = _empty_like(rho, (self.n_species, n)) if out is None else out
        energy = e is not None
        if energy and T_out is None:
            T_out = _empty_like(rho, (n,))
        args = [rho, e if energy else T, Y, T_out if energy else None, w]
        ptrs = [_ptr(a)[0] for a in args]
        _check(lib().pyro_net_production_rates_noalloc(self._h, n, ptrs[0], ptrs[1], 1 if energy else 0,
                                                       ptrs[2], ptrs[3], ptrs[4], _stream(args)))
        return (w, T_out) if energy else w

    def prepare(self, kernels: str = "all"):
        _check(lib().pyro_mech_prepare(self._h, kernels.encode()))

    def jvp(self, rho, T, Y, d_rho, d_T, d_Y, out=None):
        """d omega [N, n] = J (d_rho, d_T, d_Y)."""
        w = _empty_like(rho, (self.n_species, _n(rho))) if out is None else out
        args = [rho, T, Y, d_rho, d_T, d_Y, w]
        _check(lib().pyro_jvp(self._h, _n(rho), *[_ptr(a)[0] for a in args], _stream(args)))
        return w

    def vjp(self, rho, T, Y, omega_bar):
        """(rho_bar [n], T_bar [n], Y_bar [N, n]) = J^T omega_bar."""
        n = _n(rho)
        rb, Tb, Yb = _empty_like(rho, (n,)), _empty_like(rho, (n,)), _empty_like(rho, (self.n_species, n))
        args = [rho, T, Y, omega_bar, rb, Tb, Yb]
        _check(lib().pyro_vjp(self._h, n, *[_ptr(a)[0] for a in args], _stream(args)))
        return rb, Tb, Yb

    def jacobian(self, rho, T, Y, out=None):
        """J [(N+1)*(N+1), n]: rows (Tdot, omega), columns (T, Y), at fixed rho."""
        NP = self.n_species + 1
        J = _empty_like(rho, (NP * NP, _n(rho))) if out is None else out
        args = [rho, T, Y, J]
        _check(lib().pyro_jacobian(self._h, _n(rho), *[_ptr(a)[0] for a in args], _stream(args)))
        return J

    def transport(self, T, Y, mu=True, kappa=True, diffusivities=True):
        """Mixture-averaged (mu [n], kappa [n], D_mix [N, n]); outputs not requested are None."""
        n = _n(T)
        m_ = _empty_like(T, (n,)) if mu else None
        k_ = _empty_like(T, (n,)) if kappa else None
        d_ = _empty_like(T, (self.n_species, n)) if diffusivities else None
        arrays = [T, Y, m_, k_, d_]
        _check(lib().pyro_transport(self._h, n, *[_ptr(a)[0] for a in arrays], _stream(arrays)))
        return m_, k_, d_

    def jacobian_adiabatic(self, rho, T, Y, out=None):
        """J [N*N, n]: dS_j/dY_k (row j, column k) of S = W omega at fixed (rho, e)."""
        N = self.n_species
        J = _empty_like(rho, (N * N, _n(rho))) if out is None else out
        args = [rho, T, Y, J]
        _check(lib().pyro_jacobian_adiabatic(self._h, _n(rho), *[_ptr(a)[0] for a in args], _stream(args)))
        return J

    def cn_step(self, dt, rho, T, Y, tol=1e-12, max_newton=20, T_out=None, Y_out=None, with_iters=False):
        """One Crank-Nicolson step of dY/dt = S/rho at fixed (rho, e): (T_next [n], Y_next [N, n]
        [, Newton steps [n], -1 where the step failed])."""
        n = _n(T)
        To = _empty_like(T, (n,)) if T_out is None else T_out
        Yo = _empty_like(T, (self.n_species, n)) if Y_out is None else Y_out
        it = _empty_like(T, (n,), "int32") if with_iters else None
        arrays = [rho, T, Y, To, Yo, it]
        ptr = [_ptr(a)[0] for a in arrays]
        _check(lib().pyro_cn_step(self._h, n, float(dt), ptr[0], ptr[1], ptr[2], float(tol), int(max_newton),
                                  ptr[3], ptr[4], ptr[5], _stream(arrays)))
        return (To, Yo, it) if with_iters else (To, Yo)

    # --- learned initial guess ---------------------------------------------------
    def mlp_n_params(self) -> int:
        return lib().pyro_mlp_n_params(self._h)

    def mlp_set_params(self, params, norm4):
        p = np.ascontiguousarray(params, dtype=np.float64)
        nm = np.ascontiguousarray(norm4, dtype=np.float64)
        _check(lib().pyro_mlp_set_params(self._h, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(nm.ctypes.data)))

    def mlp_get_params(self):
        p = np.zeros(self.mlp_n_params())
        nm = np.zeros(4)
        _check(lib().pyro_mlp_get_params(self._h, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(nm.ctypes.data)))
        return p, nm

    def mlp_train(self, T, Y, options: str = "", stream=None) -> float:
        loss = ctypes.c_double()
        args = [T, Y]
        _check(lib().pyro_mlp_train(self._h, _n(T), _ptr(T)[0], _ptr(Y)[0], options.encode() if options else None,
                                    ctypes.byref(loss), _stream(args)))
        return loss.value

    def mlp_grad(self, e, Y, T):
        g = np.zeros(self.mlp_n_params())
        loss = ctypes.c_double()
        _check(lib().pyro_mlp_grad(self._h, _n(e), _ptr(e)[0], _ptr(Y)[0], _ptr(T)[0], ctypes.byref(loss),
                                   ctypes.c_void_p(g.ctypes.data)))
        return loss.value, g

    def mlp_guess(self, e, Y):
        y, Tg = _empty_like(e, (_n(e),)), _empty_like(e, (_n(e),))
        args = [e, Y, y, Tg]
        _check(lib().pyro_mlp_guess(self._h, _n(e), *[_ptr(a)[0] for a in args], _stream(args)))
        return y, Tg

    def mlp_save(self, path: str):
        _check(lib().pyro_mlp_save(self._h, path.encode()))

    def mlp_load(self, path: str):
        _check(lib().pyro_mlp_load(self._h, path.encode()))

    def nonconverged(self, stream=None) -> int:
        c = ctypes.c_int64()
        _check(lib().pyro_nonconverged(self._h, stream or ctypes.c_void_p(0), ctypes.byref(c)))
        return c.value

    def math_eval(self, fn: int, x):
        y = _empty_like(x, (_n(x),))
        args = [x, y]
        _check(lib().pyro_math_eval(self._h, int(fn), _n(x), *[_ptr(a)[0] for a in args], _stream(args)))
        return y
