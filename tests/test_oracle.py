"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an identity, a conservation law, a limit, a printed worked example, an
independent algorithm (bisection, dual-number derivatives vs finite differences), or the
data-preparation code that produced the mechanism (NASA anchor values).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth
from tests import handmech

R = 8314.462618
P0 = 101325.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    return vals


@pytest.fixture(scope="module")
def orc(mech_files):
    paths, objs = mech_files
    return {i: O.Oracle(paths[i]) for i in (0, 1)}, objs


def _states(idx, n, orc_obj):
    st = synth.config_states(idx, n=n)
    rho = orc_obj.density(st.p, st.T, st.Y)
    return st, rho


# --- Arrhenius: worked example (Sec. 2.2 / Sec. 2.3 listings) ---------------

def test_arrhenius_worked_example(tmp_path):
    g = _golden("arrhenius_worked_example.txt")
    m = handmech.abcd_mechanism(A=g["A"], b=g["b"], theta=g["theta"])
    o = O.Oracle(handmech.write(m, str(tmp_path), "arr.txt"))
    # the printed folded constant is ln A rounded to 2 decimals
    assert abs(math.log(g["A"]) - g["lnA_printed"]) <= 0.5 * 10 ** -g["lnA_printed_decimals"]
    T = np.array([300.0, 800.0, 1200.0, 2000.0, 3000.0])
    Y = np.full((4, T.size), 0.25)
    rho = np.ones_like(T)
    kf = o.reaction_data(rho, T, Y)["kf"][0]
    printed = np.exp(g["lnA_printed"] + g["b"] * np.log(T) - g["theta"] / T)
    # only the 2-decimal rounding of ln A separates the two
    assert np.all(np.abs(kf / printed - 1.0) < 6e-3)
    # and the sign/placement of b and theta: k grows with T for this example
    assert np.all(np.diff(kf) > 0)


# --- NASA-7 thermo ----------------------------------------------------------

@pytest.mark.parametrize("idx", [0, 1])
def test_nasa_derivative_identities(orc, idx):
    o = orc[0][idx]
    for k in range(o.N):
        for T in (250.0, 600.0, 999.0, 1001.0, 1500.0, 3000.0):
            cp, hRT, sR, gRT = o.species_thermo(k, T)
            dh, ds, _ = o.species_thermo_dT(k, T)
            assert abs(dh - cp) <= 1e-12 * abs(cp)          # d(h/R)/dT = cp/R
            assert abs(ds - cp / T) <= 1e-12 * abs(cp / T)  # d(s/R)/dT = cp/(R T)
            assert abs(gRT - (hRT - sR)) <= 1e-12 * max(1.0, abs(hRT), abs(sR))


@pytest.mark.parametrize("idx", [0, 1])
def test_nasa_continuity_and_anchor_values(orc, idx):
    o, mech = orc[0][idx], orc[1][idx]
    for k, s in enumerate(mech.species):
        below = o.species_thermo(k, s.t_mid * (1 - 1e-13))
        above = o.species_thermo(k, s.t_mid)
        # cp, h, s continuous across T_mid (constrained fit)
        assert np.allclose(below[:3], above[:3], rtol=1e-9, atol=1e-9)
        # anchor values the generator fitted to (independent numpy evaluation)
        cp, hRT, sR, _ = o.species_thermo(k, 298.15)
        assert abs(hRT * 298.15 - s.h298) <= 1e-8 * max(1.0, abs(s.h298))
        assert abs(sR - s.s298) <= 1e-10 * abs(s.s298)


def test_constant_cp_closed_forms(tmp_path):
    m = handmech.abcd_mechanism(a6=(1000.0, -2000.0, 500.0, 3000.0))
    o = O.Oracle(handmech.write(m, str(tmp_path), "cc.txt"))
    for k, s in enumerate(m.species):
        a1, a6, a7 = s.nasa_low[0], s.nasa_low[5], s.nasa_low[6]
        for T in (300.0, 1500.0):
            cp, hRT, sR, _ = o.species_thermo(k, T)
            assert cp == pytest.approx(a1, rel=1e-15)
            assert hRT == pytest.approx(a1 + a6 / T, rel=1e-14)
            assert sR == pytest.approx(a1 * math.log(T) + a7, rel=1e-14)


# --- mixture / EOS / internal energy / Newton --------------------------------

@pytest.mark.parametrize("idx", [0, 1])
def test_eos_ideal_gas_total_concentration(orc, idx):
    """sum_k C_k = rho sum Y/W = p/(R T) (Eq. eos with Eq. concentrations)."""
    o = orc[0][idx]
    st, rho = _states(idx, 256, o)
    ctot = rho * (st.Y / o.W[:, None]).sum(axis=0)
    assert np.allclose(ctot, st.p / (R * st.T), rtol=1e-14)


@pytest.mark.parametrize("idx", [0, 1])
def test_newton_round_trip_and_bisection(orc, idx):
    o = orc[0][idx]
    st, rho = _states(idx, 512, o)
    e, cv = o.internal_energy(st.T, st.Y, with_cv=True)
    assert np.all(cv > 0)
    T, it, bad = o.temperature(e, st.Y)
    assert bad == 0
    assert np.max(np.abs(T - st.T) / st.T) < 1e-13
    assert it.max() <= 12
    Tb = o.temperature_bisect(e, st.Y)
    assert np.max(np.abs(T - Tb) / Tb) < 1e-13


@pytest.mark.parametrize("idx", [0, 1])
def test_cv_is_energy_derivative(orc, idx):
    """c_v = de/dT (Eq. cv) against a central difference of e(T)."""
    o = orc[0][idx]
    st, _ = _states(idx, 64, o)
    h = 1e-3
    ep = o.internal_energy(st.T + h, st.Y)
    em = o.internal_energy(st.T - h, st.Y)
    _, cv = o.internal_energy(st.T, st.Y, with_cv=True)
    near = np.abs(st.T - 1000.0) < 2 * h
    fd = (ep - em) / (2 * h)
    assert np.allclose(fd[~near], cv[~near], rtol=1e-7)


def test_newton_iteration_cap_reports_failure(orc):
    o = orc[0][0]
    st, _ = _states(0, 32, o)
    e = o.internal_energy(st.T, st.Y)
    T, it, bad = o.temperature(e, st.Y, max_iter=1)
    assert bad == 32 and np.all(it == -1)


# --- kinetics ---------------------------------------------------------------

@pytest.mark.parametrize("idx", [0, 1])
def test_gibbs_equilibrium_gives_zero_net_rates(orc, idx):
    """At C_k = (p0/RT) exp(-g_k/RT + sum_e lambda_e n_ke) every reaction satisfies
    prod C^nu = K_c (element balance), so every R_j vanishes (Eq. reaction_rates,
    Eq. equil_constants): a Gibbs minimum for the implied element totals."""
    o, mech = orc[0][idx], orc[1][idx]
    els = [e for e, _ in mech.elements]
    rng = np.random.default_rng(7)
    for T in (900.0, 1500.0, 2500.0):
        lam = rng.uniform(-3.0, 3.0, size=len(els))
        gRT = np.array([o.species_thermo(k, T)[3] for k in range(o.N)])
        n_ke = np.array([[s.composition.get(e, 0) for e in els] for s in mech.species])
        lnC = math.log(P0 / (R * T)) - gRT + n_ke @ lam
        C = np.exp(lnC)
        rho = float((C * o.W).sum())
        Y = (C * o.W / rho)[:, None]
        d = o.reaction_data(np.array([rho]), np.array([T]), Y)
        Rf, Rr = d["Rf"][:, 0], d["Rr"][:, 0]
        scale = np.maximum(np.abs(Rf), np.abs(Rr))
        ok = scale > 1e-290
        assert ok.sum() > 0.5 * o.M
        assert np.all(np.abs(Rf - Rr)[ok] <= 1e-11 * scale[ok])


@pytest.mark.parametrize("idx", [0, 1])
def test_mass_and_element_conservation(orc, idx):
    o, mech = orc[0][idx], orc[1][idx]
    st, rho = _states(idx, 256, o)
    w, G = o.net_production_rates(rho, st.T, st.Y, with_gross=True)
    mass = (o.W[:, None] * w).sum(axis=0)
    assert np.all(np.abs(mass) <= 1e-14 * (o.W[:, None] * G).sum(axis=0))
    for e, _ in mech.elements:
        n_k = np.array([s.composition.get(e, 0) for s in mech.species], dtype=float)
        tot = (n_k[:, None] * w).sum(axis=0)
        assert np.all(np.abs(tot) <= 1e-14 * (n_k[:, None] * G).sum(axis=0) + 1e-300)


@pytest.mark.parametrize("idx", [0, 1, 4])
def test_mechanism_element_balance(orc, mech_files, idx):
    mech = mech_files[1][idx]
    for r in mech.reactions:
        for e, _ in mech.elements:
            lhs = sum(nu * mech.species[k].composition.get(e, 0) for k, nu in r.reactants)
            rhs = sum(nu * mech.species[k].composition.get(e, 0) for k, nu in r.products)
            assert lhs == rhs


def test_third_body_unit_efficiencies_is_total_concentration(tmp_path):
    """All eps = 1: [M] = sum C = p/(R T), so k_threebody = k_arrhenius * p/(RT)."""
    m1 = handmech.abcd_mechanism(kind="threebody")
    m2 = handmech.abcd_mechanism(kind="arrhenius")
    o1 = O.Oracle(handmech.write(m1, str(tmp_path), "tb.txt"))
    o2 = O.Oracle(handmech.write(m2, str(tmp_path), "pl.txt"))
    st = synth.generate_states(4, 16, (400.0, 2500.0), (0.5, 5.0), seed=3)
    rho = o1.density(st.p, st.T, st.Y)
    k1 = o1.reaction_data(rho, st.T, st.Y)["kf"][0]
    k2 = o2.reaction_data(rho, st.T, st.Y)["kf"][0]
    assert np.allclose(k1 / k2, st.p / (R * st.T), rtol=1e-13)


def test_falloff_limits(tmp_path):
    """Troe blending in its limits.  With x = log10 Pr + c, f = x/(n - d x) tends to
    -1/d as |x| -> inf, so log F -> log Fcent * d^2/(1 + d^2): k -> k0 [M] Fcent^0.0192...
    as [M] -> 0 and k -> k_inf Fcent^0.0192... as [M] -> inf.  At x = 0, F = Fcent.
    Lindemann (no Troe data) gives k = k_inf/2 exactly at Pr = 1."""
    A, b, th = 1e12, 0.3, 4000.0
    A0, b0, th0 = 1e16, -1.0, 1000.0
    a, T3, T1, T2 = 0.6, 100.0, 1500.0, 5000.0
    mt = handmech.abcd_mechanism(kind="falloff", A=A, b=b, theta=th, low=(A0, b0, th0),
                                 troe=(a, T3, T1, T2))
    ot = O.Oracle(handmech.write(mt, str(tmp_path), "troe.txt"))
    T = np.array([500.0, 1200.0, 2200.0])
    Y = np.full((4, 3), 0.25)
    Wm = 1.0 / (0.25 / ot.W).sum()
    kinf = A * T ** b * np.exp(-th / T)
    k0 = A0 * T ** b0 * np.exp(-th0 / T)
    Fcent = (1 - a) * np.exp(-T / T3) + a * np.exp(-T / T1) + np.exp(-T2 / T)
    d = 0.14
    Flim = Fcent ** (d * d / (1 + d * d))
    for rho_scale, expect in ((1e-30, "low"), (1e30, "high")):
        rho = np.full(3, rho_scale)
        M = rho / Wm
        kf = ot.reaction_data(rho, T, Y)["kf"][0]
        ref = (k0 * M if expect == "low" else kinf) * Flim
        assert np.allclose(kf, ref, rtol=3e-2)   # approach is O(1/log10 Pr)
    # centre of the falloff curve: log10 Pr = -c  ->  F = Fcent
    c = -0.4 - 0.67 * np.log10(Fcent)
    Pr = 10.0 ** (-c)
    rho = Pr * kinf / k0 * Wm
    kf = ot.reaction_data(rho, T, Y)["kf"][0]
    assert np.allclose(kf, kinf * Pr / (1 + Pr) * Fcent, rtol=1e-12)
    ml = handmech.abcd_mechanism(kind="falloff", A=A, b=b, theta=th, low=(A0, b0, th0))
    ol = O.Oracle(handmech.write(ml, str(tmp_path), "lind.txt"))
    M_half = kinf / k0                     # Pr = 1
    rho = M_half * Wm
    kf = ol.reaction_data(rho, T, Y)["kf"][0]
    assert np.allclose(kf, 0.5 * kinf, rtol=1e-13)


def test_irreversible_limit_and_detailed_balance(tmp_path):
    """Products far below reactants in Gibbs energy: K_c -> inf and R -> k_f prod C^nu'.
    Detailed balance: k_f/k_r = K_c and, for sum nu = 0, K_c = exp(-Delta g/RT)."""
    m = handmech.abcd_mechanism(a6=(0.0, 0.0, -5e4, -5e4))
    o = O.Oracle(handmech.write(m, str(tmp_path), "irr.txt"))
    T = np.array([400.0, 800.0])
    Y = np.full((4, 2), 0.25)
    rho = np.ones(2)
    d = o.reaction_data(rho, T, Y)
    assert np.all(d["Rr"][0] <= 1e-50 * d["Rf"][0])
    # sum nu = 0 here: K_c = exp(-(g_OH + g_O - g_H - g_O2)/RT), a closed form for const cp
    for i, t in enumerate(T):
        g = [o.species_thermo(k, t)[3] for k in range(4)]
        assert d["Kc"][0, i] == pytest.approx(math.exp(-(g[2] + g[3] - g[0] - g[1])), rel=1e-12)


@pytest.mark.parametrize("idx", [0, 1])
def test_long_double_envelope(orc, idx):
    o = orc[0][idx]
    st, rho = _states(idx, 128, o)
    w, G = o.net_production_rates(rho, st.T, st.Y, with_gross=True)
    wl = o.net_production_rates_ld(rho, st.T, st.Y)
    assert np.all(np.abs(w - wl) <= 1e-12 * G + 1e-300)


# --- derivatives --------------------------------------------------------------

def _fd_jacobian(o, rho, T, Y, h_rel=1e-7):
    """Central differences, h_c = 1e-7 * max(|x_c|, s_c) with s_T = T, s_Y = 1e-3 (reading c17)."""
    N = o.N
    NP = N + 1
    n = T.size
    J = np.zeros((NP, NP, n))
    for c in range(NP):
        Tp, Tm, Yp, Ym = T.copy(), T.copy(), Y.copy(), Y.copy()
        if c == 0:
            h = h_rel * T
            Tp = T + h; Tm = T - h
        else:
            h = h_rel * np.maximum(np.abs(Y[c - 1]), 1e-3)
            Yp[c - 1] += h; Ym[c - 1] -= h
        wp = o.net_production_rates(rho, Tp, Yp); wm = o.net_production_rates(rho, Tm, Ym)
        tp = o.temperature_rate(rho, Tp, Yp); tm = o.temperature_rate(rho, Tm, Ym)
        J[0, c] = (tp - tm) / (2 * h)
        J[1:, c] = (wp - wm) / (2 * h)
    return J


@pytest.mark.parametrize("idx", [0, 1])
def test_jacobian_vs_central_fd(orc, idx):
    o = orc[0][idx]
    n = 6 if idx == 1 else 24
    st, rho = _states(idx, n, o)
    NP = o.N + 1
    J = o.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    Jfd = _fd_jacobian(o, rho, st.T, st.Y)
    # scale entries by the row's gross magnitude: |J_rc| x_c-scale ~ row activity
    xs = np.concatenate([st.T[None], np.maximum(st.Y, 1e-3)], axis=0)   # column scales
    row = np.max(np.abs(J) * xs[None], axis=1, keepdims=True) + 1e-300
    err = np.abs(J - Jfd) * xs[None] / row
    assert np.max(err) < 1e-5


@pytest.mark.parametrize("idx", [0, 1])
def test_jacobian_first_order_fd_error_is_linear_in_delta(orc, idx):
    """The check of the paper's Jacobian section: the error of first-order forward
    differences against the Jacobian falls linearly with the step until roundoff
    takes over.  Per state, the column-scaled relative error E(delta) drops 10x
    per decade from 1e-3 to 1e-6 (truncation, slope 1).  A missing or wrong term
    in J would make E level off at the size of that term.  Below delta ~ 1e-8,
    roundoff makes E grow again (E(1e-12) > 10 E(1e-8))."""
    o = orc[0][idx]
    n = 4
    st = synth.config_states(idx, n=n, offset_seed=77)
    rho = o.density(st.p, st.T, st.Y)
    NP = o.N + 1
    J = o.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    xs = np.concatenate([st.T[None], np.maximum(st.Y, 1e-3)], axis=0)

    def rows(T, Y):
        return np.concatenate([o.temperature_rate(rho, T, Y)[None], o.net_production_rates(rho, T, Y)], axis=0)

    f0 = rows(st.T, st.Y)
    Jfd = {}
    for d in (1e-3, 1e-4, 1e-5, 1e-6, 1e-8, 1e-12):
        Jfd[d] = np.zeros_like(J)
        for c in range(NP):
            h = d * xs[c]
            T, Y = st.T.copy(), st.Y.copy()
            if c == 0:
                T = T + h
            else:
                Y[c - 1] = Y[c - 1] + h
            Jfd[d][:, c] = (rows(T, Y) - f0) / h

    def err(Jref):
        return {d: np.array([np.linalg.norm((F[:, :, i] - Jref[:, :, i]) * xs[None, :, i]) /
                             np.linalg.norm(Jref[:, :, i] * xs[None, :, i]) for i in range(n)])
                for d, F in Jfd.items()}

    E = err(J)
    for d, d10 in ((1e-3, 1e-4), (1e-4, 1e-5), (1e-5, 1e-6)):
        ratio = E[d] / E[d10]
        assert np.all((ratio > 8.0) & (ratio < 12.0)), (d, ratio)
    assert np.all(E[1e-6] < 1e-4)
    assert np.all(E[1e-12] > 10 * E[1e-8])
    # the check has teeth: a 0.1 % error in the T column levels E off
    Jbad = J.copy()
    Jbad[:, 0] *= 1.001
    Eb = err(Jbad)
    assert np.any(Eb[1e-5] / Eb[1e-6] < 8.0)


@pytest.mark.parametrize("idx", [0, 1])
def test_jvp_vjp_dot_product_identity(orc, idx):
    o = orc[0][idx]
    n = 8
    st, rho = _states(idx, n, o)
    rng = np.random.default_rng(11)
    dr, dT, dY = rng.standard_normal(n) * rho, rng.standard_normal(n) * st.T, rng.standard_normal((o.N, n)) * 1e-2
    u = rng.standard_normal((o.N, n))
    Jv = o.jvp(rho, st.T, st.Y, dr, dT, dY)
    rb, Tb, Yb = o.vjp(rho, st.T, st.Y, u)
    lhs = (u * Jv).sum(axis=0)
    rhs = rb * dr + Tb * dT + (Yb * dY).sum(axis=0)
    scale = (np.abs(u) * np.abs(Jv)).sum(axis=0) + np.abs(rb * dr) + np.abs(Tb * dT) + (np.abs(Yb * dY)).sum(axis=0)
    assert np.all(np.abs(lhs - rhs) <= 1e-11 * scale)


@pytest.mark.parametrize("idx", [0, 1])
def test_temperature_rate_conserves_energy(orc, idx):
    """e(T + Tdot dt, Y + Ydot dt) - e(T, Y) = O(dt^2) with Ydot_k = W_k omega_k / rho
    (Eq. massfrac_ode at fixed e and rho)."""
    o = orc[0][idx]
    st, rho = _states(idx, 32, o)
    w = o.net_production_rates(rho, st.T, st.Y)
    Td = o.temperature_rate(rho, st.T, st.Y)
    Yd = o.W[:, None] * w / rho
    e0, cv = o.internal_energy(st.T, st.Y, with_cv=True)
    # choose dt small relative to each point's own time scale
    tau = np.minimum(st.T / (np.abs(Td) + 1e-300), 1.0 / (np.abs(Yd).max(axis=0) + 1e-300))
    res = []
    for f in (1e-4, 1e-5):
        dt = f * tau
        e1 = o.internal_energy(st.T + Td * dt, st.Y + Yd * dt)
        res.append(np.abs(e1 - e0) / (cv * st.T))
    # residual falls ~quadratically (allow rounding floor)
    assert np.all((res[1] <= 0.05 * res[0]) | (res[1] < 1e-14))


# --- MLP model definition -------------------------------------------------------

def test_mlp_backprop_matches_complex_step():
    D, H = 11, 8
    rng = np.random.default_rng(5)
    npar = O.mlp_n_params(D, H)
    P = rng.standard_normal(npar) * 0.3
    x = rng.standard_normal((16, D))
    t = rng.standard_normal(16)
    loss, g = O.mlp_loss_grad(D, H, P, x, t)
    assert loss > 0
    for _ in range(4):
        v = rng.standard_normal(npar)
        d = O.mlp_loss_dir(D, H, P, v, x, t)
        assert d == pytest.approx(float(g @ v), rel=1e-10, abs=1e-13)


def test_mlp_forward_consistent_with_loss():
    D, H = 5, 4
    rng = np.random.default_rng(2)
    P = rng.standard_normal(O.mlp_n_params(D, H))
    x = rng.standard_normal((7, D))
    y = O.mlp_forward(D, H, P, x)
    loss, _ = O.mlp_loss_grad(D, H, P, x, np.zeros(7))
    assert loss == pytest.approx(float(np.mean(y ** 2)), rel=1e-14)


def test_malformed_mechanism_rejected(tmp_path):
    p = tmp_path / "bad.txt"
    p.write_text("pyro-mech 1\nname x\nelements 1\nelement H 1.008\nspecies 1\nspecies H 1 Q 1\n")
    with pytest.raises(ValueError):
        O.Oracle(str(p))
