"""GPU parity of the chemical Jacobian at fixed (rho, e) (Eq. chem_jacobian) and
of the Crank-Nicolson step (Sec. A.3.2, Eqs. crank_nicol_rhs to crank_nicol_jac)
against the CPU oracle, element by element on the same seeded inputs, plus
properties that hold at any size (mass and energy conservation).

Tolerances.
  Jacobian: as for the (T, Y) Jacobian, each entry within 1e-11 of its own
    gross scale W_j (GJ_jk + GJ_jT |dT/dY_k|) (the oracle's GJ, reading c15
    carried over to derivatives).
  Crank-Nicolson step: both sides converge the same Newton iteration to
    max|dY| <= 1e-12 and take one more step, so they differ by the rounding of
    the residual F(Y) = Y - c - dt/(2 rho) S(Y) propagated through the Newton
    matrix: with the source term rounded at ~1e-14 of its gross scale and
    dt |lambda| <= ~10, |dY| stays below ~1e-13; the bound 1e-10 (absolute, Y
    in [0, 1]) and 1e-10 T on the temperature leave three orders of margin.
    Newton step counts agree to within one step (the GPU solves each linear
    system by FP32 LU plus FP64 refinement, so its last updates differ at
    rounding level and the stop rule can trip one step apart).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_J = 1e-11
TOL_Y = 1e-10
TOL_T = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mechs(mech_files, dev):
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    paths, _ = mech_files
    out = {}
    for i in (0, 1):
        m = B.Mechanism(paths[i])
        m.prepare("jacobian,jacobian_adiabatic,cn")
        out[i] = (m, O.Oracle(paths[i]))
    return out


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _state(idx, n, orc, seed=0):
    st = synth.config_states(idx, n=n, offset_seed=70 + seed)
    return st, orc.density(st.p, st.T, st.Y)


# --- chemical Jacobian at fixed (rho, e) ------------------------------------------

@pytest.mark.parametrize("idx,n", [(0, 200), (1, 40)])
def test_adiabatic_jacobian_matches_oracle(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho = _state(idx, n, orc)
    N = orc.N
    J = m.jacobian_adiabatic(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(N, N, n)
    Jo = orc.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, n)
    G = orc.jacobian_adiabatic_gross(rho, st.T, st.Y).reshape(N, N, n)
    assert np.all(np.isfinite(J))
    assert np.all(np.abs(J - Jo) <= TOL_J * G + 1e-300)


def test_adiabatic_jacobian_chain_rule_and_mass_conservation_on_gpu(mechs, dev):
    """Built from the library's own (T, Y) Jacobian and species energies:
    J_jk = W_j (d omega_j/dY_k - d omega_j/dT e_k/c_v); every column sums to zero."""
    m, orc = mechs[1]
    n = 2051
    st, rho = _state(1, n, orc, seed=1)
    N, NP = orc.N, orc.N + 1
    r, T, Y = _t(rho, dev), _t(st.T, dev), _t(st.Y, dev)
    J = m.jacobian_adiabatic(r, T, Y).reshape(N, N, n)
    Jty = m.jacobian(r, T, Y).reshape(NP, NP, n)
    e, cv = m.internal_energy(T, Y, with_cv=True)
    ek = torch.stack([m.internal_energy(T, torch.nn.functional.one_hot(
        torch.full((n,), k, device=dev), N).T.contiguous().double()) for k in range(N)])
    Wt = torch.tensor(orc.W, device=dev, dtype=torch.float64)
    ref = Wt[:, None, None] * (Jty[1:, 1:] - Jty[1:, :1] * (ek / cv)[None])
    G = _t(orc.jacobian_adiabatic_gross(rho, st.T, st.Y).reshape(N, N, n), dev)
    assert ((J - ref).abs() <= TOL_J * G + 1e-300).all().item()
    colsum = J.sum(dim=0).abs() / (J.abs().sum(dim=0) + 1e-300)
    assert colsum.max().item() <= 1e-12


# --- Crank-Nicolson step --------------------------------------------------------

def _cn_case(idx, n, orc, seed=0):
    cfg = synth.CONFIGS[idx]
    st = synth.config_states(idx, n=n, offset_seed=seed)
    return st, orc.density(st.p, st.T, st.Y), cfg["dt"]


@pytest.mark.parametrize("idx,mi,n", [(6, 0, 131), (5, 1, 24)])
def test_cn_step_matches_oracle(mechs, dev, idx, mi, n):
    m, orc = mechs[mi]
    st, rho, dt = _cn_case(idx, n, orc)
    Yo, To, ito, bad = orc.cn_step(dt, rho, st.T, st.Y)
    assert bad == 0
    T1, Y1, it = m.cn_step(dt, _t(rho, dev), _t(st.T, dev), _t(st.Y, dev), with_iters=True)
    T1, Y1, it = T1.cpu().numpy(), Y1.cpu().numpy(), it.cpu().numpy()
    assert np.all(it > 0) and m.nonconverged() == 0
    assert np.max(np.abs(Y1 - Yo)) <= TOL_Y
    assert np.max(np.abs(T1 - To) / To) <= TOL_T
    assert np.max(np.abs(it - ito)) <= 1
    assert np.mean(it == ito) >= 0.5
    # the step moved the state (the comparison is not of two copies of the input)
    assert np.max(np.abs(Y1 - st.Y)) > 1e3 * TOL_Y


def test_cn_step_conservation_in_place_and_edge_cases(mechs, dev):
    m, orc = mechs[0]
    st, rho, dt = _cn_case(6, 517, orc, seed=1)
    r, T, Y = _t(rho, dev), _t(st.T, dev), _t(st.Y, dev)
    e0 = m.internal_energy(T, Y)
    T1, Y1, it = m.cn_step(dt, r, T, Y, with_iters=True)
    assert (it > 0).all().item()
    # sum_k Y_k is conserved (columns of I - h J sum to one), e by construction
    assert (Y1.sum(0) - Y.sum(0)).abs().max().item() <= 1e-13
    e1 = m.internal_energy(T1, Y1)
    assert ((e1 - e0).abs() <= 1e-12 * e0.abs() + 1e-6).all().item()
    # in place (outputs alias the inputs) gives the same bits
    T2, Y2 = T.clone(), Y.clone()
    m.cn_step(dt, r, T2, Y2, T_out=T2, Y_out=Y2)
    assert torch.equal(T2, T1) and torch.equal(Y2, Y1)
    # dt = 0 returns the input state after one Newton step plus the final one
    T0, Y0, it0 = m.cn_step(0.0, r, T, Y, with_iters=True)
    assert torch.equal(Y0, Y) and (it0 == 2).all().item()
    assert ((T0 - T).abs() <= 1e-12 * T).all().item()
    # host arrays give the same result as device arrays
    Th, Yh = m.cn_step(dt, rho, st.T, st.Y)
    assert np.array_equal(Yh, Y1.cpu().numpy()) and np.array_equal(Th, T1.cpu().numpy())
    # n = 0 and bad arguments
    z = _t(np.zeros(0), dev)
    m.cn_step(dt, z, z, _t(np.zeros((orc.N, 0)), dev))
    from paper_2503_24286_gb300.binding import PyroError
    with pytest.raises(PyroError):
        m.cn_step(-1.0, r, T, Y)
    with pytest.raises(PyroError):
        m.cn_step(dt, r, T, Y, tol=0.0)


def test_cn_step_iteration_cap_reports_failure(mechs, dev):
    """max_newton = 1 cannot meet the stop rule (it needs a step after convergence):
    every state reports -1 and the failures are counted."""
    m, orc = mechs[0]
    st, rho, dt = _cn_case(6, 64, orc, seed=2)
    m.nonconverged()
    T1, Y1, it = m.cn_step(dt, _t(rho, dev), _t(st.T, dev), _t(st.Y, dev), max_newton=1, with_iters=True)
    assert (it == -1).all().item()
    assert m.nonconverged() == 64


def test_cn_step_full_size_sampled(mechs, dev):
    """The benchmark workload (2^18 states of the 53-species mechanism, dt = 3e-41 s):
    every state converges, mass and energy are conserved, sampled states match the
    oracle."""
    m, orc = mechs[1]
    cfg = synth.CONFIGS[5]
    n = cfg["n_points"]
    T0, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 5, dev)
    rho = m.density(p, T0, Y)
    e0 = m.internal_energy(T0, Y)
    T1, Y1, it = m.cn_step(cfg["dt"], rho, T0, Y, with_iters=True)
    assert (it > 0).all().item() and m.nonconverged() == 0
    assert (Y1.sum(0) - Y.sum(0)).abs().max().item() <= 1e-13
    e1 = m.internal_energy(T1, Y1)
    assert ((e1 - e0).abs() <= 1e-12 * e0.abs() + 1e-6).all().item()
    idx = np.array([0, 1, 777, n // 2, n - 1])
    ii = torch.tensor(idx, device=dev)
    Yo, To, ito, bad = orc.cn_step(cfg["dt"], rho[ii].cpu().numpy(), T0[ii].cpu().numpy(), Y[:, ii].cpu().numpy())
    assert bad == 0
    assert np.max(np.abs(Y1[:, ii].cpu().numpy() - Yo)) <= TOL_Y
    assert np.max(np.abs(T1[ii].cpu().numpy() - To) / To) <= TOL_T


# --- chord variant (the first iterate's factorisation kept for the whole step) ---------

@pytest.fixture(scope="module")
def chord(mech_files, dev):
    from paper_2503_24286_gb300 import binding as B
    paths, _ = mech_files
    out = {}
    for i in (0, 1):
        m = B.Mechanism(paths[i], "cn_newton=chord")
        m.prepare("cn")
        out[i] = (m, O.Oracle(paths[i]))
    return out


@pytest.mark.parametrize("idx,mi,n", [(6, 0, 131), (5, 1, 24)])
def test_cn_chord_matches_oracle(chord, dev, idx, mi, n):
    """The chord iteration converges to the same Crank-Nicolson step as the oracle's
    full Newton (same residual, same stop rule; more iterations)."""
    m, orc = chord[mi]
    st, rho, dt = _cn_case(idx, n, orc)
    Yo, To, ito, bad = orc.cn_step(dt, rho, st.T, st.Y)
    assert bad == 0
    T1, Y1, it = m.cn_step(dt, _t(rho, dev), _t(st.T, dev), _t(st.Y, dev), max_newton=60, with_iters=True)
    T1, Y1, it = T1.cpu().numpy(), Y1.cpu().numpy(), it.cpu().numpy()
    assert np.all(it > 0) and m.nonconverged() == 0
    assert np.max(np.abs(Y1 - Yo)) <= TOL_Y
    assert np.max(np.abs(T1 - To) / To) <= TOL_T
    assert np.all(it >= ito - 1)


def test_cn_chord_full_size(chord, dev):
    m, orc = chord[1]
    cfg = synth.CONFIGS[5]
    n = cfg["n_points"]
    T0, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 5, dev)
    rho = m.density(p, T0, Y)
    e0 = m.internal_energy(T0, Y)
    T1, Y1, it = m.cn_step(cfg["dt"], rho, T0, Y, max_newton=60, with_iters=True)
    assert (it > 0).all().item() and m.nonconverged() == 0
    assert (Y1.sum(0) - Y.sum(0)).abs().max().item() <= 1e-13
    e1 = m.internal_energy(T1, Y1)
    assert ((e1 - e0).abs() <= 1e-12 * e0.abs() + 1e-6).all().item()
    idx = np.array([0, 4097, n - 1])
    ii = torch.tensor(idx, device=dev)
    Yo, To, ito, bad = orc.cn_step(cfg["dt"], rho[ii].cpu().numpy(), T0[ii].cpu().numpy(), Y[:, ii].cpu().numpy())
    assert bad == 0
    assert np.max(np.abs(Y1[:, ii].cpu().numpy() - Yo)) <= TOL_Y


# --- Jacobian rows from tables (the large-mechanism assembly) on 53 species -------

@pytest.fixture(scope="module")
def table53(mech_files, dev, mechs):
    from paper_2503_24286_gb300 import binding as B
    paths, _ = mech_files
    m = B.Mechanism(paths[1], "jac_rows=table")
    m.prepare("jacobian,jacobian_adiabatic,cn")
    assert m.stat("jacobian_rows_from_tables") == 1 and mechs[1][0].stat("jacobian_rows_from_tables") == 0
    return m


def test_table_rows_match_inline_rows_and_oracle(table53, mechs, dev):
    """The table-driven row assembly adds the same terms as the straight-line rows in
    another order: both Jacobians agree entry by entry to 1e-11 of the gross scale
    over several blocks with a ragged tail, and the Crank-Nicolson step built on the table rows
    matches the oracle."""
    mi, orc = mechs[1]
    mt = table53
    n = 515
    st, rho = _state(1, n, orc, seed=3)
    N, NP = orc.N, orc.N + 1
    r, T, Y = _t(rho, dev), _t(st.T, dev), _t(st.Y, dev)
    Ji, Jt = mi.jacobian(r, T, Y).reshape(NP, NP, n), mt.jacobian(r, T, Y).reshape(NP, NP, n)
    G = _t(orc.jacobian_gross(rho, st.T, st.Y)[:, 1:], dev)
    assert ((Jt - Ji).abs() <= TOL_J * G + 1e-300).all().item()
    Ai, At = mi.jacobian_adiabatic(r, T, Y).reshape(N, N, n), mt.jacobian_adiabatic(r, T, Y).reshape(N, N, n)
    Ga = _t(orc.jacobian_adiabatic_gross(rho, st.T, st.Y).reshape(N, N, n), dev)
    assert ((At - Ai).abs() <= TOL_J * Ga + 1e-300).all().item()
    st, rho, dt = _cn_case(5, 24, orc, seed=4)
    Yo, To, ito, bad = orc.cn_step(dt, rho, st.T, st.Y)
    assert bad == 0
    T1, Y1, it = mt.cn_step(dt, _t(rho, dev), _t(st.T, dev), _t(st.Y, dev), with_iters=True)
    assert np.all(it.cpu().numpy() > 0) and mt.nonconverged() == 0
    assert np.max(np.abs(Y1.cpu().numpy() - Yo)) <= TOL_Y
    assert np.max(np.abs(T1.cpu().numpy() - To) / To) <= TOL_T
