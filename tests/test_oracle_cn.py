"""Pins of the oracle's enthalpy inversion, chemical Jacobian at fixed (rho, e)
and Crank-Nicolson step (Sec. A.3.1 enthalpy variant; Eqs. crank_nicol_rhs to
chem_jacobian) against closed forms, identities, an independent linear solver,
finite differences and an independent high-accuracy ODE integration."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth
from tests import handmech

R = 8314.462618


@pytest.fixture(scope="module")
def orc(mech_files):
    paths, _ = mech_files
    return {i: O.Oracle(paths[i]) for i in (0, 1)}


def _states(idx, n, o, offset_seed=0):
    st = synth.config_states(idx, n=n, offset_seed=offset_seed)
    return st, o.density(st.p, st.T, st.Y)


# --- enthalpy and its inversion -------------------------------------------------

@pytest.mark.parametrize("idx", [0, 1])
def test_enthalpy_minus_energy_is_p_over_rho(orc, idx):
    """h - e = R T / W = p / rho (Eq. eos), at every state."""
    o = orc[idx]
    st, rho = _states(idx, 256, o)
    h = o.enthalpy(st.T, st.Y)
    e = o.internal_energy(st.T, st.Y)
    assert np.allclose(h - e, st.p / rho, rtol=1e-12, atol=0)


@pytest.mark.parametrize("idx", [0, 1])
def test_cp_is_enthalpy_derivative(orc, idx):
    o = orc[idx]
    st, _ = _states(idx, 64, o)
    d = 1e-3
    fd = (o.enthalpy(st.T + d, st.Y) - o.enthalpy(st.T - d, st.Y)) / (2 * d)
    _, cp = o.enthalpy(st.T, st.Y, with_cp=True)
    _, cv = o.internal_energy(st.T, st.Y, with_cv=True)
    near = np.abs(st.T - 1000.0) < 2 * d
    assert np.allclose(fd[~near], cp[~near], rtol=1e-7)
    # c_p - c_v = R / W
    W = 1.0 / np.sum(st.Y / o.W[:, None], axis=0)
    assert np.allclose(cp - cv, R / W, rtol=1e-12)


@pytest.mark.parametrize("idx", [0, 1])
def test_enthalpy_newton_round_trip_and_bisection(orc, idx):
    o = orc[idx]
    st, _ = _states(idx, 512, o)
    h = o.enthalpy(st.T, st.Y)
    T, it, bad = o.temperature_enthalpy(h, st.Y)
    assert bad == 0 and it.max() <= 12
    assert np.max(np.abs(T - st.T) / st.T) < 1e-13
    Tb = o.temperature_bisect_enthalpy(h, st.Y)
    assert np.max(np.abs(T - Tb) / Tb) < 1e-13


# --- chemical Jacobian at fixed (rho, e) ------------------------------------------

@pytest.mark.parametrize("idx", [0, 1])
def test_adiabatic_jacobian_vs_central_fd(orc, idx):
    """dS/dY at fixed (rho, e) by dual numbers through the T inversion, against
    central differences of S(Y) with T re-solved from e (h_k = 1e-7 max(|Y_k|, 1e-3))."""
    o = orc[idx]
    n = 4 if idx == 1 else 16
    st, rho = _states(idx, n, o, offset_seed=3)
    N = o.N
    J = o.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, n)
    e = o.internal_energy(st.T, st.Y)
    Jfd = np.zeros_like(J)
    for k in range(N):
        hk = 1e-7 * np.maximum(np.abs(st.Y[k]), 1e-3)
        Yp, Ym = st.Y.copy(), st.Y.copy()
        Yp[k] += hk
        Ym[k] -= hk
        Jfd[:, k] = (o.source_at_energy(rho, e, Yp) - o.source_at_energy(rho, e, Ym)) / (2 * hk)
    xs = np.maximum(st.Y, 1e-3)[None]                    # column scales
    row = np.max(np.abs(J) * xs, axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jfd) * xs / row) < 1e-5
    # mass conservation: sum_j S_j = 0 for every Y, so every column sums to zero
    colsum = np.abs(J.sum(axis=0)) / (np.abs(J).sum(axis=0) + 1e-300)
    assert np.max(colsum) < 1e-12


def test_adiabatic_jacobian_chain_rule_on_t_y_jacobian(orc):
    """The fixed-(rho, e) Jacobian equals W_j (d omega_j/dY_k - d omega_j/dT e_k / c_v)
    built from the (T, Y) Jacobian at fixed rho and species energies from
    finite differences of e in Y (dT/dY_k at fixed e = -(de/dY_k)/c_v)."""
    o = orc[0]
    n = 8
    st, rho = _states(0, n, o, offset_seed=4)
    N, NP = o.N, o.N + 1
    Jty = o.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    e, cv = o.internal_energy(st.T, st.Y, with_cv=True)
    dedY = np.zeros((N, n))
    for k in range(N):             # e is linear in Y: the difference is exact to rounding
        Yp = st.Y.copy()
        Yp[k] += 1.0
        dedY[k] = o.internal_energy(st.T, Yp) - e
    ref = o.W[:, None, None] * (Jty[1:, 1:] - Jty[1:, :1] * (dedY / cv)[None])
    J = o.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, n)
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(J - ref) / scale) < 1e-10


# --- dense solve ------------------------------------------------------------------

def test_solve_dense_against_lapack():
    rng = np.random.default_rng(7)
    for n in (1, 3, 10, 53):
        A = rng.standard_normal((n, n)) + n * np.eye(n) * rng.uniform(0, 1)
        b = rng.standard_normal(n)
        x = O.solve_dense(A, b)
        ref = np.linalg.solve(A, b)
        assert np.allclose(x, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    # a zero leading pivot needs the row exchange
    A = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 0.0], [3.0, 0.0, 1.0]])
    b = np.array([3.0, 2.0, 4.0])
    assert np.allclose(O.solve_dense(A, b), np.linalg.solve(A, b), rtol=1e-14)
    with pytest.raises(ZeroDivisionError):
        O.solve_dense(np.zeros((2, 2)), np.ones(2))


# --- Crank-Nicolson step ------------------------------------------------------------

def _isomer_mechanism(A, b, theta):
    """A <=> B between two isomers with identical thermochemistry: K_c = 1 and T is
    independent of the composition, so dY_A/dt = -k (Y_A - Y_B) is linear."""
    els = [("C", synth.ATOMIC_WEIGHTS["C"]), ("O", synth.ATOMIC_WEIGHTS["O"])]
    sp = [handmech.const_cp_species("A", {"C": 1, "O": 1}, 3.5, -1.3e4, 20.0),
          handmech.const_cp_species("B", {"C": 1, "O": 1}, 3.5, -1.3e4, 20.0)]
    r = synth.Reaction("arrhenius", [(0, 1)], [(1, 1)], A, b, theta)
    return synth.Mechanism("isomer", els, sp, [r])


@pytest.mark.parametrize("kdt", [0.05, 0.5, 3.0, 40.0])
def test_cn_linear_closed_form(tmp_path, kdt):
    """Y_A - Y_B decays by (1 - k dt)/(1 + k dt) per step; Y_A + Y_B is conserved."""
    A, b, theta = 3e7, 0.7, 4000.0
    o = O.Oracle(handmech.write(_isomer_mechanism(A, b, theta), str(tmp_path), "iso.txt"))
    T = np.array([900.0, 1500.0, 2200.0])
    Y = np.array([[0.9, 0.2, 0.55], [0.1, 0.8, 0.45]])
    rho = o.density(np.full(3, 2.0e5), T, Y)
    assert np.all(np.abs(rho - 1.0) > 0.05)            # the 1/rho of dY/dt = S/rho matters
    k = A * T ** b * np.exp(-theta / T)
    dt = kdt / k
    out = np.zeros_like(Y)
    for i in range(3):
        Yn, Tn, it, bad = o.cn_step(dt[i], rho[i:i + 1], T[i:i + 1], Y[:, i:i + 1])
        assert bad == 0 and 1 <= it[0] <= 6
        assert abs(Tn[0] - T[i]) <= 1e-12 * T[i]
        out[:, i] = Yn[:, 0]
    d0, d1 = Y[0] - Y[1], out[0] - out[1]
    assert np.allclose(d1, d0 * (1 - kdt) / (1 + kdt), rtol=1e-12, atol=1e-15)
    assert np.allclose(out.sum(0), Y.sum(0), rtol=0, atol=1e-15)


def test_cn_second_order_against_ode_integration(tmp_path):
    """One step's error against an independent tight integration of dY/dt = S/rho at
    fixed (rho, e) (scipy DOP853, T re-solved from e at each evaluation) falls 8x
    when dt halves: the local error of the trapezoidal rule is O(dt^3)."""
    integrate = pytest.importorskip("scipy.integrate")
    mech = handmech.abcd_mechanism(A=1e10, b=0.5, theta=5000.0, a6=(2.62e4, 0.0, 4.7e3, 3.0e4))
    o = O.Oracle(handmech.write(mech, str(tmp_path), "abcd.txt"))
    Y0 = np.array([[0.04], [0.70], [0.16], [0.10]])
    T0 = np.array([1700.0])
    rho = o.density(np.array([101325.0]), T0, Y0)
    e = o.internal_energy(T0, Y0)
    S0 = o.source_at_energy(rho, e, Y0)
    tau = 0.05 / np.max(np.abs(S0[:, 0] / rho[0]) / np.maximum(Y0[:, 0], 1e-3))

    def rhs(t, y):
        return o.source_at_energy(rho, e, y[:, None])[:, 0] / rho[0]

    errs = []
    for dt in (tau, tau / 2, tau / 4):
        ref = integrate.solve_ivp(rhs, (0.0, dt), Y0[:, 0], method="DOP853", rtol=1e-13, atol=1e-16).y[:, -1]
        Yn, Tn, it, bad = o.cn_step(dt, rho, T0, Y0)
        assert bad == 0
        errs.append(np.max(np.abs(Yn[:, 0] - ref)))
        # the step conserves mass and energy (T follows e)
        assert abs(Yn[:, 0].sum() - 1.0) < 1e-14
        assert abs(o.internal_energy(Tn, Yn)[0] - e[0]) <= 1e-12 * abs(e[0]) + 1e-9
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 9.5 and 6.5 < r2 < 9.5, errs


# --- the 160-species mechanism (the references of the large GPU tests) -------------

def test_large_mechanism_adiabatic_jacobian_and_cn_step(mech_files):
    """On the 160-species / 1100-reaction mechanism: dS/dY at fixed (rho, e) against
    central differences of S with T re-solved from e, zero column sums; the
    Crank-Nicolson step (dt = 1e-46 s) satisfies its defining equation
    Y+ - Y - dt/(2 rho) (S(Y+) + S(Y)) = 0 (Eq. crank_nicol_rhs) to rounding,
    conserves mass, and keeps e(T+, Y+) = e(T, Y)."""
    o = O.Oracle(mech_files[0][4])
    N = o.N
    st = synth.config_states(4, n=2, offset_seed=60)
    rho = o.density(st.p, st.T, st.Y)
    e = o.internal_energy(st.T, st.Y)
    J = o.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, 2)
    Jfd = np.zeros_like(J)
    for k in range(N):
        hk = 1e-7 * np.maximum(np.abs(st.Y[k]), 1e-3)
        Yp, Ym = st.Y.copy(), st.Y.copy()
        Yp[k] += hk
        Ym[k] -= hk
        Jfd[:, k] = (o.source_at_energy(rho, e, Yp) - o.source_at_energy(rho, e, Ym)) / (2 * hk)
    xs = np.maximum(st.Y, 1e-3)[None]
    row = np.max(np.abs(J) * xs, axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jfd) * xs / row) < 1e-5
    assert np.max(np.abs(J.sum(axis=0)) / (np.abs(J).sum(axis=0) + 1e-300)) < 1e-12

    dt = synth.CONFIGS[8]["dt"]
    st = synth.config_states(8, n=4, offset_seed=5)
    rho = o.density(st.p, st.T, st.Y)
    e = o.internal_energy(st.T, st.Y)
    Yn, Tn, it, bad = o.cn_step(dt, rho, st.T, st.Y)
    assert bad == 0 and np.all(it >= 2)
    assert np.max(np.abs(Yn - st.Y)) > 1e-5
    F = Yn - st.Y - dt / (2 * rho) * (o.source_at_energy(rho, e, Yn) + o.source_at_energy(rho, e, st.Y))
    assert np.max(np.abs(F)) < 1e-14
    assert np.max(np.abs(Yn.sum(axis=0) - st.Y.sum(axis=0))) < 1e-14
    assert np.max(np.abs(o.internal_energy(Tn, Yn) - e) / np.abs(e)) < 1e-13
