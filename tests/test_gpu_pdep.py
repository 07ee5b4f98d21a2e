"""GPU parity of the other pressure-dependent rate forms (SRI falloff, PLOG) on
the 53-species variant with 10 SRI and 20 PLOG reactions: net production rates
(temperature or internal-energy input) and the JVP, VJP and dense Jacobian,
against the CPU oracle on the same seeded inputs; the 2^22-state workload on
sampled states.  Tolerances as for the plain mechanism (see test_gpu_forward,
test_gpu_derivatives): omega 1e-11 of the gross scale, T 1e-10 T, derivative
entries 1e-11 of their gross scale (the oracle's GJ)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_T = 1e-10
TOL_W = 1e-11
TOL_D = 1e-11   # of each derivative entry's gross scale (the oracle's GJ)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mech(mech_files, dev):
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    paths, _ = mech_files
    m = B.Mechanism(paths[7])
    m.prepare("all")
    return m, O.Oracle(paths[7])


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


@pytest.mark.parametrize("energy", [False, True])
def test_pdep_net_production_rates_match_oracle(mech, dev, energy):
    m, orc = mech
    n = 3001
    st = synth.config_states(7, n=n, offset_seed=41)
    rho = orc.density(st.p, st.T, st.Y)
    if energy:
        e = orc.internal_energy(st.T, st.Y)
        w, T = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
        T = T.cpu().numpy()
        oT, _, bad = orc.temperature(e, st.Y)
        assert bad == 0 and m.nonconverged() == 0
        assert np.max(np.abs(T - oT) / oT) <= TOL_T
        Tref = oT
    else:
        w = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), T=_t(st.T, dev))
        Tref = st.T
    w = w.cpu().numpy()
    ow, G = orc.net_production_rates(rho, Tref, st.Y, with_gross=True)
    assert np.all(np.isfinite(w))
    assert np.max(np.abs(w - ow) / np.maximum(G, 1e-300)) <= TOL_W


def test_pdep_derivatives_match_oracle(mech, dev):
    m, orc = mech
    n = 40
    st = synth.config_states(7, n=n, offset_seed=42)
    rho = orc.density(st.p, st.T, st.Y)
    N, NP = orc.N, orc.N + 1
    rng = np.random.default_rng(5)
    dr, dT, dY = rng.standard_normal(n) * rho * 0.1, rng.standard_normal(n) * 10.0, rng.standard_normal((N, n)) * 1e-3
    g = m.jvp(*[_t(a, dev) for a in (rho, st.T, st.Y, dr, dT, dY)]).cpu().numpy()
    sc = orc.jvp_scale(rho, st.T, st.Y, dr, dT, dY)
    assert np.all(np.abs(g - orc.jvp(rho, st.T, st.Y, dr, dT, dY)) <= TOL_D * sc + 1e-300)
    u = rng.standard_normal((N, n))
    rb, Tb, Yb = (x.cpu().numpy() for x in m.vjp(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev), _t(u, dev)))
    orb, oTb, oYb = orc.vjp(rho, st.T, st.Y, u)
    scale = orc.vjp_scale(rho, st.T, st.Y, u)
    assert np.all(np.abs(rb - orb) <= TOL_D * scale[0] + 1e-300)
    assert np.all(np.abs(Tb - oTb) <= TOL_D * scale[1] + 1e-300)
    assert np.all(np.abs(Yb - oYb) <= TOL_D * scale[2:] + 1e-300)
    J = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(NP, NP, n)
    Jo = orc.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    G = orc.jacobian_gross(rho, st.T, st.Y)[:, 1:]
    assert np.all(np.abs(J - Jo) <= TOL_D * G + 1e-300)


def test_pdep_full_size_sampled(mech, dev):
    m, orc = mech
    cfg = synth.CONFIGS[7]
    n = cfg["n_points"]
    T0, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 7, dev)
    rho = m.density(p, T0, Y)
    e = m.internal_energy(T0, Y)
    w, T = m.net_production_rates(rho, Y, e=e)
    assert m.nonconverged() == 0 and torch.isfinite(w).all().item()
    idx = np.array([0, 1, 99991, n // 2, n - 1])
    ii = torch.tensor(idx, device=dev)
    r_s, e_s, Y_s = rho[ii].cpu().numpy(), e[ii].cpu().numpy(), Y[:, ii].cpu().numpy()
    oT, _, bad = orc.temperature(e_s, Y_s)
    assert np.max(np.abs(T[ii].cpu().numpy() - oT) / oT) <= TOL_T
    ow, G = orc.net_production_rates(r_s, oT, Y_s, with_gross=True)
    assert np.max(np.abs(w[:, ii].cpu().numpy() - ow) / np.maximum(G, 1e-300)) <= TOL_W
