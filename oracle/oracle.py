"""ctypes front end of the CPU oracle (``pyro_oracle.cpp``) — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares nothing with the GPU library:
it compiles its own C++ source with the host compiler and reads mechanism
files with its own parser.  All arrays are species-major (SoA): ``Y[k, p]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pyro_oracle.cpp")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libpyro_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++ -O2, OpenMP, no fast-math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.c_int64
        L.orc_load.restype = P
        L.orc_load.argtypes = [ctypes.c_char_p]
        L.orc_last_error.restype = ctypes.c_char_p
        L.orc_free.argtypes = [P]
        L.orc_info.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_mol_weights.argtypes = [P, D]
        L.orc_species_thermo.argtypes = [P, ctypes.c_int, ctypes.c_double, D]
        L.orc_species_thermo_dT.argtypes = [P, ctypes.c_int, ctypes.c_double, D]
        L.orc_density.argtypes = [P, I64, D, D, D, D]
        L.orc_internal_energy.argtypes = [P, I64, D, D, D, D]
        L.orc_temperature.restype = I64
        L.orc_temperature.argtypes = [P, I64, D, D, D, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, D, ctypes.POINTER(ctypes.c_int32)]
        L.orc_temperature_bisect.argtypes = [P, I64, D, D, ctypes.c_double, ctypes.c_double, D]
        L.orc_reaction_data.argtypes = [P, I64, D, D, D, D, D, D, D]
        L.orc_net_production_rates.argtypes = [P, I64, D, D, D, D, D]
        L.orc_net_production_rates_ld.argtypes = [P, I64, D, D, D, D]
        L.orc_temperature_rate.argtypes = [P, I64, D, D, D, D]
        L.orc_jacobian.argtypes = [P, I64, D, D, D, D]
        L.orc_jacobian_gross.argtypes = [P, I64, D, D, D, D]
        L.orc_jvp.argtypes = [P, I64, D, D, D, D, D, D, D]
        L.orc_vjp.argtypes = [P, I64, D, D, D, D, D, D, D]
        L.orc_enthalpy.argtypes = [P, I64, D, D, D, D]
        L.orc_temperature_enthalpy.restype = I64
        L.orc_temperature_enthalpy.argtypes = [P, I64, D, D, D, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, D, ctypes.POINTER(ctypes.c_int32)]
        L.orc_temperature_bisect_enthalpy.argtypes = [P, I64, D, D, ctypes.c_double, ctypes.c_double, D]
        L.orc_jacobian_adiabatic.argtypes = [P, I64, D, D, D, D]
        L.orc_source_at_energy.argtypes = [P, I64, D, D, D, D]
        L.orc_has_transport.restype = ctypes.c_int
        L.orc_has_transport.argtypes = [P]
        L.orc_species_transport.argtypes = [P, ctypes.c_int, ctypes.c_double, D]
        L.orc_binary_diffusivity.restype = ctypes.c_double
        L.orc_binary_diffusivity.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_wilke_phi.argtypes = [P, ctypes.c_double, D]
        L.orc_transport.argtypes = [P, I64, D, D, D, D, D]
        L.orc_transport_ld.argtypes = [P, I64, D, D, D, D, D]
        L.orc_solve_dense.restype = ctypes.c_int
        L.orc_solve_dense.argtypes = [ctypes.c_int, D, D]
        L.orc_cn_step.restype = I64
        L.orc_cn_step.argtypes = [P, I64, ctypes.c_double, D, D, D, ctypes.c_double, ctypes.c_int, D, D,
                                  ctypes.POINTER(ctypes.c_int32)]
        L.orc_mlp_forward.argtypes = [ctypes.c_int, ctypes.c_int, D, I64, D, D]
        L.orc_mlp_loss_grad.restype = ctypes.c_double
        L.orc_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_int, D, I64, D, D, D]
        L.orc_mlp_loss_dir.restype = ctypes.c_double
        L.orc_mlp_loss_dir.argtypes = [ctypes.c_int, ctypes.c_int, D, D, I64, D, D]
        _lib = L
    return _lib


def _d(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return lib().orc_threads()


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


class Oracle:
    """One parsed mechanism."""

    def __init__(self, path: str):
        L = lib()
        self._h = L.orc_load(path.encode())
        if not self._h:
            raise ValueError("oracle: " + L.orc_last_error().decode())
        n, m = ctypes.c_int(), ctypes.c_int()
        L.orc_info(self._h, ctypes.byref(n), ctypes.byref(m))
        self.N, self.M = n.value, m.value
        self.W = np.zeros(self.N)
        L.orc_mol_weights(self._h, _d(self.W))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_free(self._h)
            self._h = None

    # --- thermo -----------------------------------------------------------
    def species_thermo(self, k: int, T: float) -> np.ndarray:
        """[cp/R, h/RT, s/R, g/RT] of species k at T."""
        out = np.zeros(4)
        lib().orc_species_thermo(self._h, k, float(T), _d(out))
        return out

    def species_thermo_dT(self, k: int, T: float) -> np.ndarray:
        """[d(h/R)/dT, d(s/R)/dT, d(cp/R)/dT] (dual numbers)."""
        out = np.zeros(3)
        lib().orc_species_thermo_dT(self._h, k, float(T), _d(out))
        return out

    # --- mixture ----------------------------------------------------------
    def density(self, p, T, Y):
        p, T, Y = _c(p), _c(T), _c(Y)
        out = np.zeros_like(T)
        lib().orc_density(self._h, T.size, _d(p), _d(T), _d(Y), _d(out))
        return out

    def internal_energy(self, T, Y, with_cv=False):
        T, Y = _c(T), _c(Y)
        e = np.zeros_like(T)
        cv = np.zeros_like(T) if with_cv else None
        lib().orc_internal_energy(self._h, T.size, _d(T), _d(Y), _d(e), _d(cv))
        return (e, cv) if with_cv else e

    def temperature(self, e, Y, guess=None, T_guess=1200.0, tol=1e-10, max_iter=50):
        e, Y = _c(e), _c(Y)
        T = np.zeros_like(e)
        it = np.zeros(e.size, dtype=np.int32)
        g = _c(guess) if guess is not None else None
        bad = lib().orc_temperature(self._h, e.size, _d(e), _d(Y), _d(g), float(T_guess),
                                    float(tol), int(max_iter), _d(T),
                                    it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return T, it, int(bad)

    def temperature_bisect(self, e, Y, lo=100.0, hi=5000.0):
        e, Y = _c(e), _c(Y)
        T = np.zeros_like(e)
        lib().orc_temperature_bisect(self._h, e.size, _d(e), _d(Y), float(lo), float(hi), _d(T))
        return T

    def enthalpy(self, T, Y, with_cp=False):
        T, Y = _c(T), _c(Y)
        h = np.zeros_like(T)
        cp = np.zeros_like(T) if with_cp else None
        lib().orc_enthalpy(self._h, T.size, _d(T), _d(Y), _d(h), _d(cp))
        return (h, cp) if with_cp else h

    def temperature_enthalpy(self, h, Y, guess=None, T_guess=1200.0, tol=1e-10, max_iter=50):
        h, Y = _c(h), _c(Y)
        T = np.zeros_like(h)
        it = np.zeros(h.size, dtype=np.int32)
        g = _c(guess) if guess is not None else None
        bad = lib().orc_temperature_enthalpy(self._h, h.size, _d(h), _d(Y), _d(g), float(T_guess),
                                             float(tol), int(max_iter), _d(T),
                                             it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return T, it, int(bad)

    def temperature_bisect_enthalpy(self, h, Y, lo=100.0, hi=5000.0):
        h, Y = _c(h), _c(Y)
        T = np.zeros_like(h)
        lib().orc_temperature_bisect_enthalpy(self._h, h.size, _d(h), _d(Y), float(lo), float(hi), _d(T))
        return T

    # --- kinetics ---------------------------------------------------------
    def reaction_data(self, rho, T, Y):
        rho, T, Y = _c(rho), _c(T), _c(Y)
        n = T.size
        kf, Kc, Rf, Rr = (np.zeros((self.M, n)) for _ in range(4))
        lib().orc_reaction_data(self._h, n, _d(rho), _d(T), _d(Y), _d(kf), _d(Kc), _d(Rf), _d(Rr))
        return dict(kf=kf, Kc=Kc, Rf=Rf, Rr=Rr)

    def net_production_rates(self, rho, T, Y, with_gross=False):
        rho, T, Y = _c(rho), _c(T), _c(Y)
        n = T.size
        w = np.zeros((self.N, n))
        g = np.zeros((self.N, n)) if with_gross else None
        lib().orc_net_production_rates(self._h, n, _d(rho), _d(T), _d(Y), _d(w), _d(g))
        return (w, g) if with_gross else w

    def net_production_rates_ld(self, rho, T, Y):
        rho, T, Y = _c(rho), _c(T), _c(Y)
        w = np.zeros((self.N, T.size))
        lib().orc_net_production_rates_ld(self._h, T.size, _d(rho), _d(T), _d(Y), _d(w))
        return w

    def temperature_rate(self, rho, T, Y):
        rho, T, Y = _c(rho), _c(T), _c(Y)
        out = np.zeros_like(T)
        lib().orc_temperature_rate(self._h, T.size, _d(rho), _d(T), _d(Y), _d(out))
        return out

    def jacobian(self, rho, T, Y):
        """[(N+1)*(N+1), n]: rows (Tdot, omega_1..N) x columns (T, Y_1..N)."""
        rho, T, Y = _c(rho), _c(T), _c(Y)
        NP = self.N + 1
        J = np.zeros((NP * NP, T.size))
        lib().orc_jacobian(self._h, T.size, _d(rho), _d(T), _d(Y), _d(J))
        return J

    def jacobian_gross(self, rho, T, Y):
        """[N+1, N+2, n] gross scale of each derivative entry (reading c15 carried
        to derivatives): rows (Tdot, omega_1..N) x columns (rho, T, Y_1..N), the
        magnitudes of the forward and reverse rates' derivatives summed with |nu|."""
        rho, T, Y = _c(rho), _c(T), _c(Y)
        G = np.zeros(((self.N + 1) * (self.N + 2), T.size))
        lib().orc_jacobian_gross(self._h, T.size, _d(rho), _d(T), _d(Y), _d(G))
        return G.reshape(self.N + 1, self.N + 2, T.size)

    def jvp_scale(self, rho, T, Y, drho, dT, dY):
        """[N, n] per-entry scale of the JVP: sum_c GJ_kc |v_c|."""
        G = self.jacobian_gross(rho, T, Y)[1:]
        v = np.concatenate([np.abs(_c(drho))[None], np.abs(_c(dT))[None], np.abs(_c(dY))], axis=0)
        return np.einsum("kcn,cn->kn", G, v)

    def vjp_scale(self, rho, T, Y, wbar):
        """[N+2, n] per-entry scale of the VJP (rho_bar, T_bar, Y_bar): sum_k |u_k| GJ_kc."""
        G = self.jacobian_gross(rho, T, Y)[1:]
        return np.einsum("kcn,kn->cn", G, np.abs(_c(wbar)))

    def jacobian_adiabatic_gross(self, rho, T, Y):
        """[N*N, n] per-entry scale of dS_j/dY_k at fixed (rho, e):
        W_j (GJ_jk + GJ_jT |dT/dY_k|), dT/dY_k = -e_k/c_v (Eq. int_energy, Eq. cv)."""
        rho, T, Y = _c(rho), _c(T), _c(Y)
        G = self.jacobian_gross(rho, T, Y)[1:]
        _, cv = self.internal_energy(T, Y, with_cv=True)
        ek = np.zeros((self.N, T.size))
        for k in range(self.N):
            Yk = np.zeros_like(Y)
            Yk[k] = 1.0
            ek[k] = self.internal_energy(T, Yk)
        dTdY = np.abs(ek) / cv
        S = self.W[:, None, None] * (G[:, 2:] + G[:, 1:2] * dTdY[None])
        return S.reshape(self.N * self.N, T.size)

    def jacobian_adiabatic(self, rho, T, Y):
        """[N*N, n]: dS_j/dY_k (row j, column k) of S = W omega at fixed (rho, e)."""
        rho, T, Y = _c(rho), _c(T), _c(Y)
        J = np.zeros((self.N * self.N, T.size))
        lib().orc_jacobian_adiabatic(self._h, T.size, _d(rho), _d(T), _d(Y), _d(J))
        return J

    def source_at_energy(self, rho, e, Y):
        """S = W omega [N, n] with T solved from (e, Y)."""
        rho, e, Y = _c(rho), _c(e), _c(Y)
        S = np.zeros((self.N, e.size))
        lib().orc_source_at_energy(self._h, e.size, _d(rho), _d(e), _d(Y), _d(S))
        return S

    def cn_step(self, dt, rho, T, Y, tol=1e-12, max_newton=20):
        """One Crank-Nicolson step of dY/dt = S/rho at fixed (rho, e): (Y_next [N, n],
        T_next [n], Newton steps [n] (-1: failed), number failed)."""
        rho, T, Y = _c(rho), _c(T), _c(Y)
        n = T.size
        Yo, To = np.zeros((self.N, n)), np.zeros(n)
        it = np.zeros(n, dtype=np.int32)
        bad = lib().orc_cn_step(self._h, n, float(dt), _d(rho), _d(T), _d(Y), float(tol), int(max_newton),
                                _d(Yo), _d(To), it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return Yo, To, it, int(bad)

    # --- mixture-averaged transport (Sec. A.2) ---------------------------------
    @property
    def has_transport(self) -> bool:
        return bool(lib().orc_has_transport(self._h))

    def species_transport(self, k: int, T: float):
        """(mu_k, kappa_k) of species k at T."""
        out = np.zeros(2)
        lib().orc_species_transport(self._h, int(k), float(T), _d(out))
        return out[0], out[1]

    def binary_diffusivity(self, k: int, j: int, T: float) -> float:
        return lib().orc_binary_diffusivity(self._h, int(k), int(j), float(T))

    def wilke_phi(self, T: float) -> np.ndarray:
        """[N, N] Wilke's Phi_kj at T."""
        Phi = np.zeros((self.N, self.N))
        lib().orc_wilke_phi(self._h, float(T), _d(Phi))
        return Phi

    def transport(self, T, Y, long_double=False):
        """(mu [n], kappa [n], D_km [N, n]) of the mixture-averaged model."""
        T, Y = _c(T), _c(Y)
        n = T.size
        mu, kappa, Dm = np.zeros(n), np.zeros(n), np.zeros((self.N, n))
        f = lib().orc_transport_ld if long_double else lib().orc_transport
        f(self._h, n, _d(T), _d(Y), _d(mu), _d(kappa), _d(Dm))
        return mu, kappa, Dm

    def jvp(self, rho, T, Y, drho, dT, dY):
        args = [_c(a) for a in (rho, T, Y, drho, dT, dY)]
        out = np.zeros((self.N, args[1].size))
        lib().orc_jvp(self._h, args[1].size, *[_d(a) for a in args], _d(out))
        return out

    def vjp(self, rho, T, Y, wbar):
        rho, T, Y, wbar = _c(rho), _c(T), _c(Y), _c(wbar)
        n = T.size
        rb, Tb, Yb = np.zeros(n), np.zeros(n), np.zeros((self.N, n))
        lib().orc_vjp(self._h, n, _d(rho), _d(T), _d(Y), _d(wbar), _d(rb), _d(Tb), _d(Yb))
        return rb, Tb, Yb


def solve_dense(A, b):
    """x of A x = b by the oracle's Gaussian elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64, order="C")
    x = np.array(b, dtype=np.float64)
    if lib().orc_solve_dense(x.size, _d(A), _d(x)) != 0:
        raise ZeroDivisionError("singular matrix")
    return x


# --- MLP (model definition in FP64 with bf16 rounding points) -------------

def mlp_n_params(D: int, H: int) -> int:
    return H * D + H + H * H + H + H + 1


def mlp_forward(D: int, H: int, params, x):
    params, x = _c(params), _c(x)
    n = x.shape[0]
    y = np.zeros(n)
    lib().orc_mlp_forward(D, H, _d(params), n, _d(x), _d(y))
    return y


def mlp_loss_grad(D: int, H: int, params, x, t):
    params, x, t = _c(params), _c(x), _c(t)
    g = np.zeros(mlp_n_params(D, H))
    loss = lib().orc_mlp_loss_grad(D, H, _d(params), x.shape[0], _d(x), _d(t), _d(g))
    return loss, g


def mlp_loss_dir(D: int, H: int, params, v, x, t):
    params, v, x, t = _c(params), _c(v), _c(x), _c(t)
    return lib().orc_mlp_loss_dir(D, H, _d(params), _d(v), x.shape[0], _d(x), _d(t))
