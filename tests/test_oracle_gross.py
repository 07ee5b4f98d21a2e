"""Pins of the oracle's per-entry derivative scale and of its network model.

The derivative scale GJ (reading c15 carried over to derivatives) is the sum,
over the reactions of a species, of the magnitudes of the forward and reverse
rates' derivatives.  It is checked three ways, none of which reuses its code:
it bounds every entry of the oracle's Jacobian (triangle inequality), it
equals the entry's magnitude where only one rate of one reaction moves with the
variable (a one-reaction mechanism), and it agrees with the same sums assembled
here from central differences of the forward and reverse rates of progress.

The network model (D -> H -> H -> 1, SiLU, bf16 rounding points) is checked
against a forward pass worked by hand (tests/golden/mlp_tiny_network.txt).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth
from tests import handmech

R = 8314.462618
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def orc(mech_files):
    paths, objs = mech_files
    return {i: (O.Oracle(paths[i]), objs[i]) for i in (0, 1)}


def _states(idx, n, o, seed=31):
    st = synth.config_states(idx, n=n, offset_seed=seed)
    return st, o.density(st.p, st.T, st.Y)


def _nu(mech):
    """[N, M] net stoichiometric coefficients nu'' - nu' from the mechanism object."""
    nu = np.zeros((mech.n_species, mech.n_reactions))
    for j, r in enumerate(mech.reactions):
        for k, c in r.products:
            nu[k, j] += c
        for k, c in r.reactants:
            nu[k, j] -= c
    return nu


@pytest.mark.parametrize("idx", [0, 1])
def test_gross_bounds_every_derivative_entry(orc, idx):
    o, _ = orc[idx]
    n = 16 if idx == 0 else 4
    st, rho = _states(idx, n, o)
    G = o.jacobian_gross(rho, st.T, st.Y)                        # [N+1, N+2, n]
    NP = o.N + 1
    J = o.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)           # columns T, Y
    assert np.all(G >= 0)
    assert np.all(np.abs(J) <= G[:, 1:] * (1 + 1e-12) + 1e-300)
    # rho column of the production rates, by a JVP along rho
    jr = o.jvp(rho, st.T, st.Y, np.ones(n), np.zeros(n), np.zeros((o.N, n)))
    assert np.all(np.abs(jr) <= G[1:, 0] * (1 + 1e-12) + 1e-300)
    # the bound is not vacuous: for most entries it is within a few orders of |J|
    big = G[1:, 1:] > 0
    ratio = np.abs(J[1:])[big] / G[1:, 1:][big]
    assert np.median(ratio) > 1e-3


@pytest.mark.parametrize("reversible", [True, False])
def test_gross_equals_magnitude_for_one_reaction(tmp_path, reversible):
    """H + O2 <=> OH + O alone.  A Y column of a reactant moves only the forward
    rate, so GJ equals |J| there; with the reaction irreversible, every column of
    every production rate moves one rate only and GJ = |J| throughout."""
    m = handmech.abcd_mechanism()
    m.reactions[0].reversible = reversible
    o = O.Oracle(handmech.write(m, str(tmp_path), "one.txt"))
    st = synth.generate_states(4, 12, (500.0, 2500.0), (0.5, 5.0), seed=8)
    rho = o.density(st.p, st.T, st.Y)
    n = st.T.size
    G = o.jacobian_gross(rho, st.T, st.Y)
    J = o.jacobian(rho, st.T, st.Y).reshape(5, 5, n)
    # reactant columns Y_H (species 0) and Y_O2 (species 1)
    for c in (0, 1):
        assert np.allclose(np.abs(J[1:, 1 + c]), G[1:, 2 + c], rtol=1e-12, atol=0)
    if not reversible:
        assert np.allclose(np.abs(J[1:]), G[1:, 1:], rtol=1e-12, atol=0)
        jr = o.jvp(rho, st.T, st.Y, np.ones(n), np.zeros(n), np.zeros((4, n)))
        assert np.allclose(np.abs(jr), G[1:, 0], rtol=1e-12, atol=0)
    else:
        # both rates move with T: GJ = |nu| (|dRf/dT| + |dRr/dT|) > |J| unless their
        # derivatives have opposite signs
        d = o.reaction_data(rho, st.T, st.Y)
        assert np.all(d["Rr"][0] > 0)
        assert np.all(G[1:, 1] >= np.abs(J[1:, 0]) * (1 - 1e-12))


@pytest.mark.parametrize("idx,n", [(0, 5), (1, 2)])
def test_gross_from_central_differences_of_the_rates(orc, idx, n):
    """GJ assembled here from central differences of Rf and Rr (each reaction,
    each variable) with the mechanism object's stoichiometry, and the Tdot row
    from the species energies, the gross scale of omega and differences of c_v."""
    o, mech = orc[idx]
    st, rho = _states(idx, n, o, seed=33)
    N, M = o.N, o.M
    nu = np.abs(_nu(mech))
    G = o.jacobian_gross(rho, st.T, st.Y)
    scale = [rho, st.T] + [np.maximum(st.Y[k], 1e-3) for k in range(N)]
    Gfd = np.zeros((N, N + 2, n))
    dcv = np.zeros((N + 2, n))

    def ev(c, h):
        r, T, Y = rho.copy(), st.T.copy(), st.Y.copy()
        if c == 0:
            r = r + h
        elif c == 1:
            T = T + h
        else:
            Y[c - 2] = Y[c - 2] + h
        d = o.reaction_data(r, T, Y)
        _, cv = o.internal_energy(T, Y, with_cv=True)
        return d["Rf"], d["Rr"], r * cv

    for c in range(N + 2):
        h = 1e-6 * scale[c]
        fp, rp, cp_ = ev(c, h)
        fm, rm, cm = ev(c, -h)
        dRf, dRr = (fp - fm) / (2 * h), (rp - rm) / (2 * h)
        Gfd[:, c] = nu @ (np.abs(dRf) + np.abs(dRr))
        dcv[c] = (cp_ - cm) / (2 * h)
    rows = np.max(Gfd * np.array(scale)[None], axis=1, keepdims=True)
    err = np.abs(Gfd - G[1:]) * np.array(scale)[None]
    assert np.all(err <= 1e-6 * rows + 1e-300)
    # temperature-rate row
    _, Gw = o.net_production_rates(rho, st.T, st.Y, with_gross=True)
    _, cv = o.internal_energy(st.T, st.Y, with_cv=True)
    th = np.array([[o.species_thermo(k, t) for t in st.T] for k in range(N)])   # [N, n, 4]
    eh = R * st.T[None] * (th[:, :, 1] - 1.0)
    deh = R * (th[:, :, 0] - 1.0)
    rcv = rho * cv
    Tg = (np.abs(eh) * Gw).sum(0) / rcv
    G0 = (np.abs(eh)[:, None] * Gfd).sum(0) / rcv + Tg * np.abs(dcv) / rcv
    G0[1] += (np.abs(deh) * Gw).sum(0) / rcv
    assert np.allclose(G0, G[0], rtol=1e-6, atol=0)


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    return vals


def test_mlp_forward_tiny_network_by_hand():
    """The network model on a 2-2-2-1 net worked by hand: bf16 rounding of the
    inputs (ties to even), SiLU = z / (1 + e^-z), bf16 rounding of both hidden
    layers, no rounding of the output, row-major weights (row = output unit)."""
    g = _golden("mlp_tiny_network.txt")
    D, H = int(g["D"]), int(g["H"])
    W1 = [g["W1_00"], g["W1_01"], g["W1_10"], g["W1_11"]]
    b1 = [g["b1_0"], math.log(3.0) + g["b1_1_minus_ln3"]]
    W2 = [g["W2_00"], g["W2_01"], g["W2_10"], g["W2_11"]]
    b2 = [g["b2_0"], g["b2_1"]]
    P = np.array(W1 + b1 + W2 + b2 + [g["w3_0"], g["w3_1"], g["b3"]])
    x = np.array([[g["x0"], g["x1"]]])
    y = O.mlp_forward(D, H, P, x)
    assert y[0] == pytest.approx(g["y"], abs=1e-15)
    # the inputs are rounded before use (a nudge that keeps x_0's bf16 value keeps
    # y), and the pin sees the weight layout (a transposed first layer moves y)
    assert abs(O.mlp_forward(D, H, P, np.array([[1.0 + 3 * 2 ** -8 + 1e-9, 1.0]]))[0] - g["y"]) < 1e-15
    Pt = P.copy()
    Pt[0:4] = [W1[0], W1[2], W1[1], W1[3]]
    assert abs(O.mlp_forward(D, H, Pt, x)[0] - g["y"]) > 1e-5


@pytest.mark.parametrize("lnPr", [-46.0, 0.0, 46.0, 69.0])
def test_falloff_blend_derivative_at_extreme_pr(tmp_path, lnPr):
    """Lindemann falloff H + O2 (+M) <=> OH + O with an inert N2 that enters only
    [M]: with k = k_inf Pr/(1+Pr), Pr = k0 [M]/k_inf, the derivative of the rate
    of progress R = k P (P = C_H C_O2 - C_OH C_O/K_c) along Y_N2 is
    dR/dY_N2 = R/([M] (1 + Pr)) * rho/W_N2 in closed form.  The oracle's
    derivatives must reproduce it from Pr = 1e-20 to Pr = 1e30 (where 1 - Pr/(1+Pr)
    cancels to nothing in floating point)."""
    A, b, th, A0, b0, th0 = 1e12, 0.3, 4000.0, 1e16, -1.0, 1000.0
    m = handmech.abcd_mechanism(kind="falloff", A=A, b=b, theta=th, low=(A0, b0, th0))
    m.species.append(handmech.const_cp_species("N2", {"N": 2}, 3.5, 0.0, 23.0))
    m.elements.append(("N", synth.ATOMIC_WEIGHTS["N"]))
    o = O.Oracle(handmech.write(m, str(tmp_path), "lind_inert.txt"))
    T = np.array([800.0, 1500.0])
    Y = np.array([[0.1, 0.2], [0.2, 0.1], [0.15, 0.25], [0.05, 0.15], [0.5, 0.3]])
    Wm = 1.0 / (Y / o.W[:, None]).sum(axis=0)
    kinf = A * T ** b * np.exp(-th / T)
    k0 = A0 * T ** b0 * np.exp(-th0 / T)
    M = math.exp(lnPr) * kinf / k0              # [M] that puts Pr at e^lnPr
    rho = M * Wm
    d = o.reaction_data(rho, T, Y)
    R_ = d["Rf"][0] - d["Rr"][0]
    Pr = k0 * M / kinf
    expect = R_ / (M * (1.0 + Pr)) * rho / o.W[4]
    e4 = np.zeros((5, 2))
    e4[4] = 1.0
    dw = o.jvp(rho, T, Y, np.zeros(2), np.zeros(2), e4)     # d omega / d Y_N2
    assert np.allclose(dw[0], -expect, rtol=1e-12, atol=0)  # omega_H = -R
    assert np.allclose(dw[2], expect, rtol=1e-12, atol=0)   # omega_OH = +R
    assert np.all(dw[4] == 0.0)


@pytest.mark.parametrize("Y_O", [1e-75, 1e-100, 1e-200])
def test_jacobian_entry_closed_form_at_tiny_mass_fractions(tmp_path, Y_O):
    """Recombination 2 O (+M) <=> O2, Lindemann falloff, with O and O2 both far
    below any finite-difference or complex step (as at equilibrium states, where
    mass fractions reach 1e-200).  At fixed (rho, T):
      d omega_O2/d Y_O = k 2 C_O rho/W_O + dk/d[M] rho/W_O (C_O^2 - C_O2/K_c),
      dk/d[M] = k0/(1 + Pr)^2  (k = k_inf Pr/(1+Pr), Pr = k0 [M]/k_inf),
    and d omega_O/d Y_O = -2 of it.  Evaluated here from the Arrhenius constants;
    the oracle's Jacobian must reproduce it to rounding.  A complex step of 1e-30
    fails this by many orders of magnitude (its h^2 term dominates)."""
    A, b, th, A0, b0, th0 = 1e10, 0.5, 5000.0, 1e16, -1.0, 1000.0
    m = handmech.abcd_mechanism(kind="falloff", A=A, b=b, theta=th, low=(A0, b0, th0))
    m.reactions[0].reactants = [(3, 2)]
    m.reactions[0].products = [(1, 1)]
    o = O.Oracle(handmech.write(m, str(tmp_path), "two_o.txt"))
    T, rho = np.array([1500.0, 900.0]), np.array([0.8, 3.0])
    Y = np.array([[0.3, 0.2], [Y_O ** 2, Y_O * 1e-30], [0.7, 0.8], [Y_O, Y_O]])
    C = rho * Y / o.W[:, None]
    M = C.sum(axis=0)
    kinf = A * T ** b * np.exp(-th / T)
    k0 = A0 * T ** b0 * np.exp(-th0 / T)
    Pr = k0 * M / kinf
    k = kinf * Pr / (1.0 + Pr)
    Kc = o.reaction_data(rho, T, Y)["Kc"][0]
    expect = (k * 2.0 * C[3] + k0 / (1.0 + Pr) ** 2 * (C[3] ** 2 - C[1] / Kc)) * rho / o.W[3]
    J = o.jacobian(rho, T, Y).reshape(5, 5, 2)       # rows (Tdot, omega), columns (T, Y)
    assert np.allclose(J[2, 4], expect, rtol=1e-13, atol=0)
    assert np.allclose(J[4, 4], -2.0 * expect, rtol=1e-13, atol=0)


def test_jvp_is_linear_at_states_with_tiny_mass_fractions(orc):
    """The JVP is the linear map J v: at states whose mass fractions reach 1e-200
    it must stay additive in v and reproduce the
    Jacobian's columns along unit directions."""
    o, _ = orc[1]
    st, rho = _states(1, 3, o, seed=35)
    Y = st.Y.copy()
    Y[:10] = 10.0 ** -np.arange(150.0, 250.0, 10.0)[:, None]
    Y /= Y.sum(axis=0, keepdims=True)
    rng = np.random.default_rng(36)
    v1 = [rng.standard_normal(3) * rho * 0.1, rng.standard_normal(3) * 10.0, rng.standard_normal((o.N, 3)) * 1e-3]
    v2 = [rng.standard_normal(3) * rho * 0.1, rng.standard_normal(3) * 10.0, rng.standard_normal((o.N, 3)) * 1e-3]
    j1, j2 = o.jvp(rho, st.T, Y, *v1), o.jvp(rho, st.T, Y, *v2)
    j12 = o.jvp(rho, st.T, Y, *[a + b for a, b in zip(v1, v2)])
    sc = o.jvp_scale(rho, st.T, Y, *[np.abs(a) + np.abs(b) for a, b in zip(v1, v2)])
    assert np.all(np.abs(j12 - j1 - j2) <= 1e-13 * sc + 1e-300)
    NP = o.N + 1
    J = o.jacobian(rho, st.T, Y).reshape(NP, NP, 3)
    for c in (0, 1, 5, 12):                     # T and three mass fractions (two of them tiny)
        dT = np.full(3, 1.0 if c == 0 else 0.0)
        dY = np.zeros((o.N, 3))
        if c > 0:
            dY[c - 1] = 1.0
        assert np.array_equal(o.jvp(rho, st.T, Y, np.zeros(3), dT, dY), J[1:, c])


def test_jvp_bounded_by_gross_scale_at_equilibrium_states(orc):
    """At Gibbs-minimised equilibrium states (mass fractions down to ~1e-230) the
    JVP obeys the triangle inequality |J v|_k <= sum_c GJ_kc |v_c| entry by entry."""
    from tests.edge_states import equilibrium_states
    o, mech = orc[1]
    rho, T, Y = equilibrium_states(o, mech, 40, seed=17)
    rng = np.random.default_rng(18)
    n = T.size
    dr, dT, dY = rng.standard_normal(n) * rho * 0.1, rng.standard_normal(n) * 10.0, rng.standard_normal((o.N, n)) * 1e-3
    j = o.jvp(rho, T, Y, dr, dT, dY)
    sc = o.jvp_scale(rho, T, Y, dr, dT, dY)
    assert np.all(np.abs(j) <= sc * (1 + 1e-12) + 1e-300)
