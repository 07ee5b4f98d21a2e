"""GPU derivative kernels (JVP, VJP, dense Jacobian) against the CPU oracle's
dual-number (forward-mode) derivatives, against central finite differences, and against each
other (u.(J v) = (J^T u).v).  Also the torch.autograd.Function wrapper.

Tolerance: each entry is compared element by element at 1e-11 of its own
gross scale (reading c15 carried over to derivatives): for d omega_k/d x_c the
oracle's GJ_kc = sum_j |nu_kj| (|d Rf_j/d x_c| + |d Rr_j/d x_c|), the sizes of
the forward and reverse terms that cancel in that entry; the JVP takes
sum_c GJ_kc |v_c|, the VJP sum_k |u_k| GJ_kc, the Tdot row the same magnitudes
through its product and quotient rules.  A wrong or missing term of a minor
species or a single reaction is then visible in its own entry.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


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
        m.prepare("all")
        out[i] = (m, O.Oracle(paths[i]))
    return out


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _state(idx, n, orc, seed=0):
    st = synth.config_states(idx, n=n, offset_seed=50 + seed)
    rho = orc.density(st.p, st.T, st.Y)
    return st, rho


@pytest.mark.parametrize("idx,n", [(0, 300), (1, 48)])
def test_jvp_matches_oracle(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho = _state(idx, n, orc)
    rng = np.random.default_rng(3)
    dr = rng.standard_normal(n) * rho * 0.1
    dT = rng.standard_normal(n) * 10.0
    dY = rng.standard_normal((orc.N, n)) * 1e-3
    g = m.jvp(*[_t(a, dev) for a in (rho, st.T, st.Y, dr, dT, dY)]).cpu().numpy()
    ref = orc.jvp(rho, st.T, st.Y, dr, dT, dY)
    scale = orc.jvp_scale(rho, st.T, st.Y, dr, dT, dY)
    assert np.all(np.isfinite(g))
    assert np.all(np.abs(g - ref) <= TOL * scale + 1e-300)


@pytest.mark.parametrize("idx,n", [(0, 300), (1, 48)])
def test_vjp_matches_oracle(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho = _state(idx, n, orc, seed=1)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((orc.N, n))
    rb, Tb, Yb = (x.cpu().numpy() for x in m.vjp(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev), _t(u, dev)))
    orb, oTb, oYb = orc.vjp(rho, st.T, st.Y, u)
    scale = orc.vjp_scale(rho, st.T, st.Y, u)                       # [N+2, n]
    assert np.all(np.abs(rb - orb) <= TOL * scale[0] + 1e-300)
    assert np.all(np.abs(Tb - oTb) <= TOL * scale[1] + 1e-300)
    assert np.all(np.abs(Yb - oYb) <= TOL * scale[2:] + 1e-300)


@pytest.mark.parametrize("idx,n", [(0, 200), (1, 40)])
def test_jacobian_matches_oracle(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho = _state(idx, n, orc, seed=2)
    NP = orc.N + 1
    J = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(NP, NP, n)
    Jo = orc.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    G = orc.jacobian_gross(rho, st.T, st.Y)[:, 1:]                  # columns T, Y
    assert np.all(np.isfinite(J))
    assert np.all(np.abs(J - Jo) <= TOL * G + 1e-300)


def test_jacobian_central_differences_on_gpu(mechs, dev):
    """Central FD of the GPU's own omega and Tdot (h = 1e-7 relative) vs the GPU Jacobian."""
    m, orc = mechs[1]
    n = 64
    st, rho = _state(1, n, orc, seed=3)
    NP = orc.N + 1
    J = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(NP, NP, n)
    W = orc.W

    def rows(T, Y):
        tr, tT, tY = _t(rho, dev), _t(T, dev), _t(Y, dev)
        w = m.net_production_rates(tr, tY, T=tT).cpu().numpy()
        e_, cv = m.internal_energy(tT, tY, with_cv=True)
        # Tdot = -sum_k (h_k - R T) omega_k / (rho c_v); h_k - R T = W_k (e_k) per unit mass
        # evaluated with the library's internal energy of pure species
        eh = np.zeros_like(w)
        for k in range(orc.N):
            Yk = np.zeros_like(Y); Yk[k] = 1.0
            eh[k] = m.internal_energy(tT, _t(Yk, dev)).cpu().numpy() * W[k]
        Td = -(eh * w).sum(axis=0) / (rho * cv.cpu().numpy())
        return np.concatenate([Td[None], w], axis=0)
    xs = np.concatenate([st.T[None], np.maximum(st.Y, 1e-3)], axis=0)
    Jfd = np.zeros_like(J)
    for c in range(NP):
        h = 1e-7 * xs[c]
        Tp, Tm, Yp, Ym = st.T.copy(), st.T.copy(), st.Y.copy(), st.Y.copy()
        if c == 0:
            Tp += h; Tm -= h
        else:
            Yp[c - 1] += h; Ym[c - 1] -= h
        Jfd[:, c] = (rows(Tp, Yp) - rows(Tm, Ym)) / (2 * h)
    row = np.max(np.abs(J) * xs[None], axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(J - Jfd) * xs[None] / row) <= 1e-5


def test_jvp_vjp_dot_identity_and_jacobian_column(mechs, dev):
    m, orc = mechs[1]
    n = 2048
    st, rho = _state(1, n, orc, seed=4)
    rng = np.random.default_rng(9)
    T, Y, r = _t(st.T, dev), _t(st.Y, dev), _t(rho, dev)
    dr, dT, dY = _t(rng.standard_normal(n) * rho * 0.1, dev), _t(rng.standard_normal(n) * 5, dev), \
        _t(rng.standard_normal((orc.N, n)) * 1e-3, dev)
    u = _t(rng.standard_normal((orc.N, n)), dev)
    Jv = m.jvp(r, T, Y, dr, dT, dY)
    rb, Tb, Yb = m.vjp(r, T, Y, u)
    lhs = (u * Jv).sum(0)
    rhs = rb * dr + Tb * dT + (Yb * dY).sum(0)
    scale = (u.abs() * Jv.abs()).sum(0) + (rb * dr).abs() + (Tb * dT).abs() + (Yb * dY).abs().sum(0)
    assert ((lhs - rhs).abs() <= 1e-10 * scale).all().item()
    # the Jacobian's T column equals the JVP along T
    NP = orc.N + 1
    J = m.jacobian(r, T, Y).reshape(NP, NP, n)
    one, zero = torch.ones_like(T), torch.zeros_like(T)
    jt = m.jvp(r, T, Y, zero, one, torch.zeros_like(Y))
    sc = J[1:, 0].abs() + jt.abs() + 1e-300
    assert ((J[1:, 0] - jt).abs() <= 1e-11 * sc.max(dim=0).values).all().item()


def test_autograd_function(mechs, dev):
    from paper_2503_24286_gb300.autograd import net_production_rates
    m, orc = mechs[0]
    n = 256
    st, rho = _state(0, n, orc, seed=5)
    r = _t(rho, dev).requires_grad_(True)
    T = _t(st.T, dev).requires_grad_(True)
    Y = _t(st.Y, dev).requires_grad_(True)
    w = net_production_rates(m, r, T, Y)
    u = torch.randn_like(w)
    (w * u).sum().backward()
    rb, Tb, Yb = m.vjp(r.detach(), T.detach(), Y.detach(), u)
    assert torch.equal(r.grad, rb) and torch.equal(T.grad, Tb) and torch.equal(Y.grad, Yb)
    # forward mode through torch.autograd.forward_ad (dual tensors)
    import torch.autograd.forward_ad as fwAD
    dr, dT, dY = torch.randn_like(r) * 0.01, torch.randn_like(T), torch.randn_like(Y) * 1e-3
    with fwAD.dual_level():
        out = net_production_rates(m, fwAD.make_dual(r.detach(), dr), fwAD.make_dual(T.detach(), dT),
                                   fwAD.make_dual(Y.detach(), dY))
        tang = fwAD.unpack_dual(out).tangent
    ref = m.jvp(r.detach(), T.detach(), Y.detach(), dr, dT, dY)
    assert torch.equal(tang, ref)


def test_derivatives_full_size_sampled(mechs, dev):
    """2^20 states (the derivative workload): Jacobian and VJP on the GPU, sampled
    points against the oracle, everything finite."""
    m, orc = mechs[1]
    n = synth.CONFIGS[2]["n_points"]
    T0, p, Y = synth.generate_states_torch(53, n, synth.CONFIGS[2]["T"], synth.CONFIGS[2]["p_atm"],
                                           synth.STATE_SEED_BASE + 2, dev)
    rho = m.density(p, T0, Y)
    NP = 54
    J = m.jacobian(rho, T0, Y)
    assert torch.isfinite(J).all().item()
    idx = np.array([0, 1, 12345, n // 2, n - 1])
    ii = torch.tensor(idx, device=dev)
    Js = J[:, ii].cpu().numpy().reshape(NP, NP, -1)
    Ts, Ys, rs = T0[ii].cpu().numpy(), Y[:, ii].cpu().numpy(), rho[ii].cpu().numpy()
    Jo = orc.jacobian(rs, Ts, Ys).reshape(NP, NP, -1)
    G = orc.jacobian_gross(rs, Ts, Ys)[:, 1:]
    assert np.all(np.abs(Js - Jo) <= TOL * G + 1e-300)
    del J
    u = torch.randn((53, n), dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    rb, Tb, Yb = m.vjp(rho, T0, Y, u)
    assert torch.isfinite(Yb).all().item() and torch.isfinite(Tb).all().item()
    us = u[:, ii].cpu().numpy()
    orb, oTb, oYb = orc.vjp(rs, Ts, Ys, us)
    scale = orc.vjp_scale(rs, Ts, Ys, us)
    assert np.all(np.abs(Tb[ii].cpu().numpy() - oTb) <= TOL * scale[1])
    assert np.all(np.abs(Yb[:, ii].cpu().numpy() - oYb) <= TOL * scale[2:] + 1e-300)


@pytest.mark.parametrize("idx", [0, 1, 7, "7-mixed"])
def test_warp_per_state_jvp_vjp_match_oracle(mech_files, mixed_reversibility_mech, dev, idx):
    """The warp-per-state JVP and VJP kernels (variant=warp: lanes split the
    reactions, species adjoints gathered per species) against the oracle, every
    entry within 1e-11 of its gross scale, over several blocks with a ragged tail
    (7-mixed: every third reaction irreversible)."""
    from paper_2503_24286_gb300 import binding as B
    paths, _ = mech_files
    path = mixed_reversibility_mech if idx == "7-mixed" else paths[idx]
    idx = 7 if idx == "7-mixed" else idx
    mw = B.Mechanism(path, "variant=warp")
    assert mw.stat("deriv_warp_per_state") == 1
    orc = O.Oracle(path)
    n = 203
    st, rho = _state(idx, n, orc, seed=7)
    rng = np.random.default_rng(13)
    dr, dT, dY = rng.standard_normal(n) * rho * 0.1, rng.standard_normal(n) * 10.0, rng.standard_normal((orc.N, n)) * 1e-3
    u = rng.standard_normal((orc.N, n))
    g = mw.jvp(*[_t(a, dev) for a in (rho, st.T, st.Y, dr, dT, dY)]).cpu().numpy()
    assert np.all(np.isfinite(g))
    ref = orc.jvp(rho, st.T, st.Y, dr, dT, dY)
    assert np.all(np.abs(g - ref) <= TOL * orc.jvp_scale(rho, st.T, st.Y, dr, dT, dY) + 1e-300)
    rb, Tb, Yb = (x.cpu().numpy() for x in mw.vjp(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev), _t(u, dev)))
    orb, oTb, oYb = orc.vjp(rho, st.T, st.Y, u)
    sc = orc.vjp_scale(rho, st.T, st.Y, u)
    assert np.all(np.abs(rb - orb) <= TOL * sc[0] + 1e-300)
    assert np.all(np.abs(Tb - oTb) <= TOL * sc[1] + 1e-300)
    assert np.all(np.abs(Yb - oYb) <= TOL * sc[2:] + 1e-300)
