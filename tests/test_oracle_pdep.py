"""Pins of the oracle's other pressure-dependent rate forms (the paper names
"additional potential pressure dependencies" next to Troe in Sec. A.1 without
formulas; the standard SRI falloff and PLOG forms are taken, readings p1, p2):

* SRI: with a exp(-b/T) + exp(-T/c) = 1, d = 1, e = 0 it is the Lindemann form
  exactly; at Pr = 1 (X = 1) F = d [a exp(-b/T) + exp(-T/c)] T^e in closed form;
  for |log10 Pr| -> inf, F -> d T^e with |ln F - ln(d T^e)| <= |ln base| X;
* PLOG: at a node pressure k is that node's Arrhenius value; below the first and
  above the last node it is the end node's; ln k is linear in ln p inside a
  segment and continuous across nodes; identical nodes make k independent of p;
* the 53-species mechanism with SRI and PLOG reactions conserves mass and
  elements, vanishes at a Gibbs-minimised equilibrium, and its (dual-number)
  Jacobian agrees with central differences.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth
from tests import handmech

R = 8314.462618
P0 = 101325.0


def _arr(A, b, th, T):
    return A * T ** b * np.exp(-th / T)


def test_sri_lindemann_centre_and_limits(tmp_path):
    A, b, th = 1e12, 0.3, 4000.0
    A0, b0, th0 = 1e16, -1.0, 1000.0
    T = np.array([500.0, 1200.0, 2200.0])
    Y = np.full((4, 3), 0.25)
    # base = 1 (c -> 0 removes exp(-T/c)), d = 1, e = 0: Lindemann
    ms = handmech.abcd_mechanism(kind="falloff", A=A, b=b, theta=th, low=(A0, b0, th0))
    ms.reactions[0].sri = (1.0, 0.0, 1e-30)
    os_ = O.Oracle(handmech.write(ms, str(tmp_path), "sri1.txt"))
    ol = O.Oracle(handmech.write(handmech.abcd_mechanism(kind="falloff", A=A, b=b, theta=th, low=(A0, b0, th0)),
                                 str(tmp_path), "lind.txt"))
    for rho in (1e-3, 1.0, 1e3):
        r = np.full(3, rho)
        assert np.allclose(os_.reaction_data(r, T, Y)["kf"][0], ol.reaction_data(r, T, Y)["kf"][0], rtol=1e-15)
    # general SRI at the centre Pr = 1 and in the limits
    a, bb, c, d, e = 0.7, 600.0, 900.0, 1.3, 0.2
    ms.reactions[0].sri = (a, bb, c, d, e)
    o = O.Oracle(handmech.write(ms, str(tmp_path), "sri2.txt"))
    Wm = 1.0 / (0.25 / o.W).sum()
    kinf, k0 = _arr(A, b, th, T), _arr(A0, b0, th0, T)
    base = a * np.exp(-bb / T) + np.exp(-T / c)
    rho = kinf / k0 * Wm                      # [M] = rho / Wm makes Pr = 1
    kf = o.reaction_data(rho, T, Y)["kf"][0]
    assert np.allclose(kf, 0.5 * kinf * d * base * T ** e, rtol=1e-12)
    for scale in (1e-30, 1e30):
        rho = scale * kinf / k0 * Wm
        M = rho / Wm
        Pr = k0 * M / kinf
        kf = o.reaction_data(rho, T, Y)["kf"][0]
        F = kf / (kinf * Pr / (1 + Pr))
        X = 1.0 / (1.0 + np.log10(Pr) ** 2)
        assert np.all(np.abs(np.log(F) - np.log(d * T ** e)) <= np.abs(np.log(base)) * X * (1 + 1e-9) + 1e-13)


def _plog_mech(nodes):
    m = handmech.abcd_mechanism()
    m.reactions[0].kind = "plog"
    m.reactions[0].plog = nodes
    return m


def _rho_for_p(o, p, T, Y):
    return o.density(p, T, Y)


def test_plog_nodes_ends_linearity_and_continuity(tmp_path):
    nodes = [(0.1 * P0, 1e11, 0.2, 3000.0), (1.0 * P0, 3e12, -0.1, 5000.0), (10.0 * P0, 2e12, 0.4, 4000.0)]
    o = O.Oracle(handmech.write(_plog_mech(nodes), str(tmp_path), "plog.txt"))
    T = np.array([700.0, 1500.0, 2600.0])
    Y = np.full((4, 3), 0.25)

    def k_at(p):
        pp = np.full(3, p)
        return o.reaction_data(_rho_for_p(o, pp, T, Y), T, Y)["kf"][0]
    for pn, A, b, th in nodes:
        assert np.allclose(k_at(pn), _arr(A, b, th, T), rtol=1e-12)
    assert np.allclose(k_at(0.01 * P0), _arr(*nodes[0][1:], T), rtol=1e-14)
    assert np.allclose(k_at(1000.0 * P0), _arr(*nodes[-1][1:], T), rtol=1e-14)
    # ln k linear in ln p within the second segment: equal steps in ln p give equal steps in ln k
    ps = np.exp(np.linspace(math.log(1.5 * P0), math.log(8.0 * P0), 3))
    lk = np.log(np.array([k_at(p) for p in ps]))
    assert np.allclose(lk[2] - lk[1], lk[1] - lk[0], rtol=1e-9, atol=1e-12)
    # continuity at the interior node
    eps = 1e-9
    assert np.allclose(k_at(P0 * (1 - eps)), k_at(P0 * (1 + eps)), rtol=1e-7)
    # identical nodes: no pressure dependence
    same = [(0.1 * P0, 1e11, 0.2, 3000.0), (3.0 * P0, 1e11, 0.2, 3000.0), (30.0 * P0, 1e11, 0.2, 3000.0)]
    o2 = O.Oracle(handmech.write(_plog_mech(same), str(tmp_path), "plog2.txt"))
    for p in (0.05 * P0, 0.7 * P0, 5.0 * P0, 50.0 * P0):
        pp = np.full(3, p)
        k = o2.reaction_data(o2.density(pp, T, Y), T, Y)["kf"][0]
        assert np.allclose(k, _arr(1e11, 0.2, 3000.0, T), rtol=1e-13)


@pytest.fixture(scope="module")
def pdep(mech_files):
    paths, objs = mech_files
    return O.Oracle(paths[7]), objs[7]


def test_pdep_mechanism_conservation_and_equilibrium(pdep):
    o, mech = pdep
    assert sum(r.kind == "plog" for r in mech.reactions) == 20
    assert sum(r.sri is not None for r in mech.reactions) == 10
    st = synth.config_states(7, n=256)
    rho = o.density(st.p, st.T, st.Y)
    w, G = o.net_production_rates(rho, st.T, st.Y, with_gross=True)
    assert np.all(np.abs((o.W[:, None] * w).sum(0)) <= 1e-14 * (o.W[:, None] * G).sum(0))
    for e, _ in mech.elements:
        n_k = np.array([s.composition.get(e, 0) for s in mech.species], dtype=float)
        assert np.all(np.abs((n_k[:, None] * w).sum(0)) <= 1e-14 * (n_k[:, None] * G).sum(0) + 1e-300)
    # Gibbs-minimised state: every forward and reverse rate balance
    els = [e for e, _ in mech.elements]
    rng = np.random.default_rng(3)
    for T in (1000.0, 2200.0):
        lam = rng.uniform(-3.0, 3.0, size=len(els))
        gRT = np.array([o.species_thermo(k, T)[3] for k in range(o.N)])
        n_ke = np.array([[s.composition.get(e, 0) for e in els] for s in mech.species])
        C = np.exp(math.log(P0 / (R * T)) - gRT + n_ke @ lam)
        rho_e = float((C * o.W).sum())
        d = o.reaction_data(np.array([rho_e]), np.array([T]), (C * o.W / rho_e)[:, None])
        Rf, Rr = d["Rf"][:, 0], d["Rr"][:, 0]
        scale = np.maximum(np.abs(Rf), np.abs(Rr))
        ok = scale > 1e-290
        assert np.all(np.abs(Rf - Rr)[ok] <= 1e-11 * scale[ok])


def test_pdep_jacobian_vs_central_fd(pdep):
    from tests.test_oracle import _fd_jacobian
    o, _ = pdep
    n = 5
    st = synth.config_states(7, n=n, offset_seed=4)
    rho = o.density(st.p, st.T, st.Y)
    NP = o.N + 1
    J = o.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    Jfd = _fd_jacobian(o, rho, st.T, st.Y)
    xs = np.concatenate([st.T[None], np.maximum(st.Y, 1e-3)], axis=0)
    row = np.max(np.abs(J) * xs[None], axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jfd) * xs[None] / row) < 1e-5
