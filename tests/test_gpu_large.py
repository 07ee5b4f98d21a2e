"""The large synthetic mechanism (160 species, 1100 reactions): the emitted
thread-per-point kernels with the per-state species arrays in a global scratch
and the species accumulators in the output arrays, against the oracle --
forward (temperature input and energy input), JVP and VJP (recomputed
intermediates, no stored Jacobian) -- plus the full-size workload sampled."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = 1e-11
TOL_D = 1e-9


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def large(mech_files, dev):
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    m = B.Mechanism(mech_files[0][4])
    m.prepare("all")
    return m, O.Oracle(mech_files[0][4])


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def test_storage_mode(large):
    m, orc = large
    assert (m.n_species, m.n_reactions) == (160, 1100)
    assert m.stat("omega_store_global") == 1 and m.stat("accumulators_in_memory") == 1


def test_large_forward_parity(large, dev):
    m, orc = large
    st = synth.config_states(4, n=300)
    rho = orc.density(st.p, st.T, st.Y)
    e = orc.internal_energy(st.T, st.Y)
    w = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), T=_t(st.T, dev)).cpu().numpy()
    ow, G = orc.net_production_rates(rho, st.T, st.Y, with_gross=True)
    assert np.all(np.abs(w - ow) <= TOL_W * G + 1e-300)
    w2, T2 = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
    oT, _, bad = orc.temperature(e, st.Y)
    assert bad == 0 and m.nonconverged() == 0
    assert np.max(np.abs(T2.cpu().numpy() - oT) / oT) <= 1e-10
    ow2, G2 = orc.net_production_rates(rho, oT, st.Y, with_gross=True)
    assert np.all(np.abs(w2.cpu().numpy() - ow2) <= TOL_W * G2 + 1e-300)


def test_large_jvp_vjp_parity(large, dev):
    m, orc = large
    n = 12
    st = synth.config_states(4, n=n, offset_seed=5)
    rho = orc.density(st.p, st.T, st.Y)
    rng = np.random.default_rng(1)
    dr, dT, dY = rng.standard_normal(n) * rho * 0.1, rng.standard_normal(n) * 5, rng.standard_normal((160, n)) * 1e-3
    u = rng.standard_normal((160, n))
    g = m.jvp(*[_t(a, dev) for a in (rho, st.T, st.Y, dr, dT, dY)]).cpu().numpy()
    rb, Tb, Yb = (x.cpu().numpy() for x in m.vjp(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev), _t(u, dev)))
    # oracle d omega/d(rho, T, Y) by complex-step JVPs along unit directions
    J = np.zeros((160, 162, n))
    for c in range(162):
        e_ = np.zeros((162, n))
        e_[c] = 1.0
        J[:, c] = orc.jvp(rho, st.T, st.Y, e_[0], e_[1], e_[2:])
    v = np.concatenate([dr[None], dT[None], dY], axis=0)
    ref = np.einsum("kcn,cn->kn", J, v)
    assert np.all(np.abs(g - ref) <= TOL_D * np.einsum("kcn,cn->kn", np.abs(J), np.abs(v)) + 1e-300)
    refb = np.einsum("kcn,kn->cn", J, u)
    sc = np.einsum("kcn,kn->cn", np.abs(J), np.abs(u))
    assert np.all(np.abs(rb - refb[0]) <= TOL_D * sc[0] + 1e-300)
    assert np.all(np.abs(Tb - refb[1]) <= TOL_D * sc[1] + 1e-300)
    assert np.all(np.abs(Yb - refb[2:]) <= TOL_D * sc[2:] + 1e-300)


def test_large_jacobian_refused(large, dev):
    from paper_2503_24286_gb300 import binding as B
    m, orc = large
    st = synth.config_states(4, n=4)
    with pytest.raises(B.PyroError) as ei:
        m.jacobian(_t(np.ones(4), dev), _t(st.T, dev), _t(st.Y, dev))
    assert ei.value.code == B.PYRO_EINVAL


def test_large_full_size_sampled(large, dev):
    m, orc = large
    n = synth.CONFIGS[4]["n_points"]
    cfg = synth.CONFIGS[4]
    T0, p, Y = synth.generate_states_torch(160, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 4, dev)
    rho = m.density(p, T0, Y)
    e = m.internal_energy(T0, Y)
    w, T = m.net_production_rates(rho, Y, e=e)
    torch.cuda.synchronize()
    assert m.nonconverged() == 0 and torch.isfinite(w).all().item()
    assert (torch.abs(T - T0) / T0).max().item() <= 1e-12
    idx = np.array([0, 7, 99999, n // 3, n - 1])
    ii = torch.tensor(idx, device=dev)
    Ys, es, rs = Y[:, ii].cpu().numpy(), e[ii].cpu().numpy(), rho[ii].cpu().numpy()
    oT, _, bad = orc.temperature(es, Ys)
    ow, G = orc.net_production_rates(rs, oT, Ys, with_gross=True)
    assert bad == 0
    assert np.all(np.abs(w[:, ii].cpu().numpy() - ow) <= TOL_W * G + 1e-300)


def test_large_warp_variant(large, dev, mech_files):
    """Warp per state on the large mechanism: oracle parity, and the same results as
    the thread-per-state kernels on the full-size workload."""
    from paper_2503_24286_gb300 import binding as B
    m, orc = large
    mw = B.Mechanism(mech_files[0][4], "variant=warp")
    st = synth.config_states(4, n=300, offset_seed=2)
    rho = orc.density(st.p, st.T, st.Y)
    e = orc.internal_energy(st.T, st.Y)
    w, T = mw.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
    oT, _, _ = orc.temperature(e, st.Y)
    ow, G = orc.net_production_rates(rho, oT, st.Y, with_gross=True)
    assert mw.nonconverged() == 0
    assert np.max(np.abs(T.cpu().numpy() - oT) / oT) <= 1e-10
    assert np.all(np.abs(w.cpu().numpy() - ow) <= TOL_W * G + 1e-300)
    n = 2 ** 16
    cfg = synth.CONFIGS[4]
    T0, p, Y = synth.generate_states_torch(160, n, cfg["T"], cfg["p_atm"], 99, dev)
    r = m.density(p, T0, Y)
    ww = mw.net_production_rates(r, Y, T=T0)
    wt = m.net_production_rates(r, Y, T=T0)
    scale = wt.abs().amax(dim=0, keepdim=True) + 1e-300
    assert ((ww - wt).abs() <= 1e-9 * scale).all().item()
