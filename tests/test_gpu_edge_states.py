"""GPU parity at the method's edge states, against the CPU oracle, every entry
within 1e-11 of its gross scale (reading c15; for derivatives the oracle's GJ):

* Gibbs-minimised equilibrium states (Eq. reaction_rates, Eq. equil_constants):
  C_k = (p0/RT) exp(-g_k/RT + sum_e lambda_e n_ke) makes every reaction satisfy
  prod C^nu = K_c, so every R_j vanishes and the kernels' forward and reverse
  activity products cancel exactly in exact arithmetic.  The net rates must
  vanish to the gross scale and the derivatives must match the oracle there.
* Falloff limits: p = 1e-4 atm and 1e4 atm push P_r = k_0 [M] / k_inf towards 0
  and infinity for every Troe and SRI reaction.
* Lindemann falloff (falloff data without Troe or SRI constants, F = 1): the
  53-species mechanism with its Troe data removed.

The equilibrium states span mass fractions down to ~1e-230, so some rates and
their derivatives fall near the bottom of the double range.  The kernels and
the oracle form the same products in different orders (e.g. kk E_i rho a_j on
the GPU against k_f C_i C_j in the oracle), and an intermediate that one of them
takes through the subnormal range (below 2.2e-308) loses its relative
precision there; derivative entries are compared with an absolute floor of
1e-250 added to 1e-11 of their gross scale (DER_FLOOR), far below any entry that
matters (a floor of 1e-290 fails at such entries).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth
from tests.edge_states import equilibrium_states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 8314.462618
P0 = 101325.0
TOL = 1e-11
DER_FLOOR = 1e-250


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mechs(mech_files, dev, tmp_path_factory):
    """{name: (library handle, oracle, mechanism object)} for the 10- and
    53-species mechanisms, the SRI/PLOG variant and the Lindemann variant."""
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    paths, objs = mech_files
    lind = synth.config_mechanism(1)
    nfall = 0
    for r in lind.reactions:
        if r.kind == "falloff":
            r.troe, r.sri = None, None
            nfall += 1
    assert nfall == 25
    lp = str(tmp_path_factory.mktemp("lind") / "lindemann53.txt")
    synth.write_mechanism(lind, lp)
    out = {}
    for name, p, obj in (("h2", paths[0], objs[0]), ("gri", paths[1], objs[1]), ("pdep", paths[7], objs[7]),
                         ("lind", lp, lind)):
        m = B.Mechanism(p)
        m.prepare("jvp,vjp,jacobian")
        out[name] = (m, O.Oracle(p), obj)
    return out


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _check_forward(m, o, rho, T, Y, dev):
    w = m.net_production_rates(_t(rho, dev), _t(Y, dev), T=_t(T, dev)).cpu().numpy()
    ow, G = o.net_production_rates(rho, T, Y, with_gross=True)
    assert np.all(np.isfinite(w))
    assert np.all(np.abs(w - ow) <= TOL * G + 1e-300)
    return w, G


def _check_derivatives(m, o, rho, T, Y, dev, seed):
    n = T.size
    rng = np.random.default_rng(seed)
    dr, dT, dY = rng.standard_normal(n) * rho * 0.1, rng.standard_normal(n) * 10.0, \
        rng.standard_normal((o.N, n)) * 1e-3
    tr, tT, tY = _t(rho, dev), _t(T, dev), _t(Y, dev)
    g = m.jvp(tr, tT, tY, _t(dr, dev), _t(dT, dev), _t(dY, dev)).cpu().numpy()
    assert np.all(np.abs(g - o.jvp(rho, T, Y, dr, dT, dY)) <= TOL * o.jvp_scale(rho, T, Y, dr, dT, dY) + DER_FLOOR)
    u = rng.standard_normal((o.N, n))
    rb, Tb, Yb = (x.cpu().numpy() for x in m.vjp(tr, tT, tY, _t(u, dev)))
    orb, oTb, oYb = o.vjp(rho, T, Y, u)
    sc = o.vjp_scale(rho, T, Y, u)
    assert np.all(np.abs(rb - orb) <= TOL * sc[0] + DER_FLOOR)
    assert np.all(np.abs(Tb - oTb) <= TOL * sc[1] + DER_FLOOR)
    assert np.all(np.abs(Yb - oYb) <= TOL * sc[2:] + DER_FLOOR)
    NP = o.N + 1
    J = m.jacobian(tr, tT, tY).cpu().numpy().reshape(NP, NP, n)
    Jo = o.jacobian(rho, T, Y).reshape(NP, NP, n)
    G = o.jacobian_gross(rho, T, Y)[:, 1:]
    assert np.all(np.isfinite(J))
    assert np.all(np.abs(J - Jo) <= TOL * G + DER_FLOOR)


@pytest.mark.parametrize("name,n", [("h2", 96), ("gri", 40), ("pdep", 24)])
def test_gibbs_equilibrium_states(mechs, dev, name, n):
    m, o, mech = mechs[name]
    rho, T, Y = equilibrium_states(o, mech, n, seed=17)
    w, G = _check_forward(m, o, rho, T, Y, dev)
    # every rate of progress vanishes: omega is zero to the gross scale on the GPU too
    assert np.all(np.abs(w) <= TOL * G + 1e-300)
    assert np.median(G) > 0
    _check_derivatives(m, o, rho, T, Y, dev, seed=18)


@pytest.mark.parametrize("name", ["gri", "pdep", "lind"])
@pytest.mark.parametrize("p_atm", [1e-4, 1e4])
def test_falloff_pressure_limits(mechs, dev, name, p_atm):
    m, o, _ = mechs[name]
    n = 64
    st = synth.generate_states(o.N, n, (300.0, 2800.0), (p_atm, p_atm), seed=int(19 + math.log10(p_atm)))
    rho = o.density(st.p, st.T, st.Y)
    _check_forward(m, o, rho, st.T, st.Y, dev)
    _check_derivatives(m, o, rho[:24], st.T[:24], st.Y[:, :24], dev, seed=20)


def test_lindemann_mechanism(mechs, dev):
    """Falloff without blending constants (F = 1) at the workload's pressures, with
    the internal-energy input (Newton) and all derivative kernels."""
    m, o, _ = mechs["lind"]
    n = 1025
    st = synth.config_states(1, n=n, offset_seed=21)
    rho = o.density(st.p, st.T, st.Y)
    e = o.internal_energy(st.T, st.Y)
    w, T = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
    oT, _, bad = o.temperature(e, st.Y)
    assert bad == 0 and m.nonconverged() == 0
    assert np.max(np.abs(T.cpu().numpy() - oT) / oT) <= 1e-10
    ow, G = o.net_production_rates(rho, oT, st.Y, with_gross=True)
    assert np.all(np.abs(w.cpu().numpy() - ow) <= TOL * G + 1e-300)
    _check_derivatives(m, o, rho[:32], st.T[:32], st.Y[:, :32], dev, seed=22)
