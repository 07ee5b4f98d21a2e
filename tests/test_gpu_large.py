"""The large synthetic mechanism (160 species, 1100 reactions): the emitted
thread-per-point kernels with the per-state species arrays in a global scratch
and the species accumulators in the output arrays, against the oracle --
forward (temperature input and energy input), JVP and VJP (recomputed
intermediates, no stored Jacobian), the dense 161 x 161 Jacobian, dS/dY at fixed
(rho, e) and the Crank-Nicolson step (Jacobian rows assembled from tables) --
plus the full-size workload sampled."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = 1e-11
TOL_D = 1e-11   # of each derivative entry's gross scale (the oracle's GJ)


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
    m.prepare("jvp,vjp,jacobian,jacobian_adiabatic,cn")
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
    ref = orc.jvp(rho, st.T, st.Y, dr, dT, dY)
    sc = orc.jvp_scale(rho, st.T, st.Y, dr, dT, dY)
    assert np.all(np.abs(g - ref) <= TOL_D * sc + 1e-300)
    orb, oTb, oYb = orc.vjp(rho, st.T, st.Y, u)
    sc = orc.vjp_scale(rho, st.T, st.Y, u)
    assert np.all(np.abs(rb - orb) <= TOL_D * sc[0] + 1e-300)
    assert np.all(np.abs(Tb - oTb) <= TOL_D * sc[1] + 1e-300)
    assert np.all(np.abs(Yb - oYb) <= TOL_D * sc[2:] + 1e-300)


def test_large_jacobian_matches_oracle(large, dev):
    """Dense d(Tdot, omega)/d(T, Y), 161 x 161 per state, rows from tables, species
    arrays in the global scratch: against the oracle's dual-number Jacobian, each
    entry within 1e-11 of its gross scale."""
    m, orc = large
    assert m.stat("jacobian_rows_from_tables") == 1 and m.stat("deriv_store_global") == 1
    n, NP = 12, 161
    st = synth.config_states(4, n=n, offset_seed=50)
    rho = orc.density(st.p, st.T, st.Y)
    J = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(NP, NP, n)
    Jo = orc.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    G = orc.jacobian_gross(rho, st.T, st.Y)[:, 1:]
    assert np.all(np.isfinite(J))
    assert np.all(np.abs(J - Jo) <= TOL_D * G + 1e-300)


def test_large_adiabatic_jacobian_oracle_chain_rule_and_columns(large, dev):
    """dS/dY at fixed (rho, e), 160 x 160: against the oracle on a few states, and on
    more states than one block (ragged tail) against the chain rule applied to the
    library's own (T, Y) Jacobian, W_j (d omega_j/dY_k - d omega_j/dT e_k/c_v);
    columns sum to zero (mass conservation)."""
    m, orc = large
    N, NP = 160, 161
    st = synth.config_states(4, n=8, offset_seed=51)
    rho = orc.density(st.p, st.T, st.Y)
    J = m.jacobian_adiabatic(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(N, N, 8)
    Jo = orc.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, 8)
    G = orc.jacobian_adiabatic_gross(rho, st.T, st.Y).reshape(N, N, 8)
    assert np.all(np.abs(J - Jo) <= TOL_D * G + 1e-300)
    n = 193
    st = synth.config_states(4, n=n, offset_seed=52)
    rho = orc.density(st.p, st.T, st.Y)
    r, T, Y = _t(rho, dev), _t(st.T, dev), _t(st.Y, dev)
    Ja = m.jacobian_adiabatic(r, T, Y).reshape(N, N, n)
    Jty = m.jacobian(r, T, Y).reshape(NP, NP, n)
    e, cv = m.internal_energy(T, Y, with_cv=True)
    ek = torch.stack([m.internal_energy(T, torch.nn.functional.one_hot(
        torch.full((n,), k, device=dev), N).T.contiguous().double()) for k in range(N)])
    Wt = torch.tensor(orc.W, device=dev, dtype=torch.float64)
    ref = Wt[:, None, None] * (Jty[1:, 1:] - Jty[1:, :1] * (ek / cv)[None])
    xt = torch.clamp(Y, min=1e-3)[None]
    rw = (ref.abs() * xt).amax(dim=1, keepdim=True) + 1e-300
    assert ((Ja - ref).abs() * xt / rw).max().item() <= 1e-11
    colsum = Ja.sum(dim=0).abs() / (Ja.abs().sum(dim=0) + 1e-300)
    assert colsum.max().item() <= 1e-12


def test_large_cn_step_matches_oracle(large, dev):
    """One Crank-Nicolson step on the 160-species mechanism (dt = 1e-46 s, T in
    [2000, 2800] K): 160 x 160 Newton systems, two states per block of the batched
    solve; against the oracle's step."""
    m, orc = large
    cfg = synth.CONFIGS[8]
    st = synth.config_states(8, n=16)
    rho = orc.density(st.p, st.T, st.Y)
    Yo, To, ito, bad = orc.cn_step(cfg["dt"], rho, st.T, st.Y)
    assert bad == 0
    T1, Y1, it = m.cn_step(cfg["dt"], _t(rho, dev), _t(st.T, dev), _t(st.Y, dev), with_iters=True)
    T1, Y1, it = T1.cpu().numpy(), Y1.cpu().numpy(), it.cpu().numpy()
    assert np.all(it > 0) and m.nonconverged() == 0
    assert np.max(np.abs(Y1 - Yo)) <= 1e-10
    assert np.max(np.abs(T1 - To) / To) <= 1e-10
    assert np.max(np.abs(it - ito)) <= 1
    assert np.max(np.abs(Y1 - st.Y)) > 1e-4
    assert m.stat("cn_solve_warps") == 2


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


def test_large_warp_jvp_vjp_parity(large, dev, mech_files):
    """Warp-per-state JVP and VJP on the 160-species mechanism (the large-mechanism
    derivative kernels: intermediates recomputed per reaction, nothing stored):
    against the oracle entry by entry, and against the thread-per-state kernels on
    2^14 states."""
    from paper_2503_24286_gb300 import binding as B
    m, orc = large
    mw = B.Mechanism(mech_files[0][4], "variant=warp")
    n = 37
    st = synth.config_states(4, n=n, offset_seed=9)
    rho = orc.density(st.p, st.T, st.Y)
    rng = np.random.default_rng(2)
    dr, dT, dY = rng.standard_normal(n) * rho * 0.1, rng.standard_normal(n) * 5, rng.standard_normal((160, n)) * 1e-3
    u = rng.standard_normal((160, n))
    g = mw.jvp(*[_t(a, dev) for a in (rho, st.T, st.Y, dr, dT, dY)]).cpu().numpy()
    assert np.all(np.abs(g - orc.jvp(rho, st.T, st.Y, dr, dT, dY)) <=
                  TOL_D * orc.jvp_scale(rho, st.T, st.Y, dr, dT, dY) + 1e-300)
    rb, Tb, Yb = (x.cpu().numpy() for x in mw.vjp(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev), _t(u, dev)))
    orb, oTb, oYb = orc.vjp(rho, st.T, st.Y, u)
    sc = orc.vjp_scale(rho, st.T, st.Y, u)
    assert np.all(np.abs(rb - orb) <= TOL_D * sc[0] + 1e-300)
    assert np.all(np.abs(Tb - oTb) <= TOL_D * sc[1] + 1e-300)
    assert np.all(np.abs(Yb - oYb) <= TOL_D * sc[2:] + 1e-300)
    # the two kernel families agree on many states (same inputs, different summation order)
    n = 2 ** 14
    cfg = synth.CONFIGS[4]
    T0, p, Y = synth.generate_states_torch(160, n, cfg["T"], cfg["p_atm"], 98, dev)
    r = m.density(p, T0, Y)
    gen = torch.Generator(device=dev).manual_seed(4)
    v = [torch.randn(n, dtype=torch.float64, device=dev, generator=gen) * r * 1e-3,
         torch.randn(n, dtype=torch.float64, device=dev, generator=gen),
         torch.randn((160, n), dtype=torch.float64, device=dev, generator=gen) * 1e-4]
    jw, jt = mw.jvp(r, T0, Y, *v), m.jvp(r, T0, Y, *v)
    sc = jt.abs().amax(dim=0, keepdim=True) + 1e-300
    assert torch.isfinite(jw).all().item() and ((jw - jt).abs() <= 1e-9 * sc).all().item()


def test_large_block_per_state_jacobians(large, dev, mech_files):
    """The dense Jacobians with one block of 8 warps per state (variant=warp: the
    per-reaction partials in shared memory, rows written once from balanced
    gathers): d(Tdot, omega)/d(T, Y) and dS/dY at fixed (rho, e) against the
    oracle entry by entry; on 600 states (more than one resident grid) against
    the thread-per-state kernels."""
    from paper_2503_24286_gb300 import binding as B
    m, orc = large
    mw = B.Mechanism(mech_files[0][4], "variant=warp")
    assert mw.stat("jacobian_cta") == 1 and mw.stat("wjac_row_groups") >= 2
    N, NP, n = 160, 161, 6
    st = synth.config_states(4, n=n, offset_seed=53)
    rho = orc.density(st.p, st.T, st.Y)
    r, T, Y = _t(rho, dev), _t(st.T, dev), _t(st.Y, dev)
    J = mw.jacobian(r, T, Y).cpu().numpy().reshape(NP, NP, n)
    assert np.all(np.abs(J - orc.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)) <=
                  TOL_D * orc.jacobian_gross(rho, st.T, st.Y)[:, 1:] + 1e-300)
    Ja = mw.jacobian_adiabatic(r, T, Y).cpu().numpy().reshape(N, N, n)
    assert np.all(np.abs(Ja - orc.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, n)) <=
                  TOL_D * orc.jacobian_adiabatic_gross(rho, st.T, st.Y).reshape(N, N, n) + 1e-300)
    n = 600
    cfg = synth.CONFIGS[4]
    T0, p, Y0 = synth.generate_states_torch(160, n, cfg["T"], cfg["p_atm"], 97, dev)
    r0 = m.density(p, T0, Y0)
    Jw, Jt = mw.jacobian(r0, T0, Y0).reshape(NP, NP, n), m.jacobian(r0, T0, Y0).reshape(NP, NP, n)
    sc = Jt.abs().amax(dim=1, keepdim=True) + 1e-300
    assert torch.isfinite(Jw).all().item() and ((Jw - Jt).abs() <= 1e-9 * sc).all().item()
