"""Dense Jacobians with one block of 8 warps per state (variant=warp): the
(T, Y) Jacobian of (Tdot, omega) at fixed rho (Eq. jacobian) and dS/dY at fixed
(rho, e) (Eq. chem_jacobian), against the oracle's dual-number derivatives,
every entry within 1e-11 of its gross scale (the tolerance of the other
derivative tests), over a persistent grid with more states than resident
blocks; host-array calls give the device-array results bit for bit; the
columns of dS/dY sum to zero (mass conservation).
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
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _handle(mech_files, mixed, idx):
    from paper_2503_24286_gb300 import binding as B
    path = mixed if idx == "7-mixed" else mech_files[0][idx]
    m = B.Mechanism(path, "variant=warp")
    assert m.stat("jacobian_cta") == 1 and m.stat("jacobian_adiabatic_cta") == 1
    return m, O.Oracle(path), (7 if idx == "7-mixed" else idx)


@pytest.mark.parametrize("idx,n", [(0, 1237), (1, 40), (7, 24), ("7-mixed", 24)])
def test_block_per_state_jacobian_matches_oracle(mech_files, mixed_reversibility_mech, dev, idx, n):
    m, orc, ci = _handle(mech_files, mixed_reversibility_mech, idx)
    st = synth.config_states(ci, n=n, offset_seed=61)
    rho = orc.density(st.p, st.T, st.Y)
    NP = orc.N + 1
    J = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(NP, NP, n)
    assert np.all(np.isfinite(J))
    Jo = orc.jacobian(rho, st.T, st.Y).reshape(NP, NP, n)
    G = orc.jacobian_gross(rho, st.T, st.Y)[:, 1:]                  # columns T, Y
    assert np.all(np.abs(J - Jo) <= TOL * G + 1e-300)


@pytest.mark.parametrize("idx,n", [(0, 1237), (1, 40), (7, 24), ("7-mixed", 24)])
def test_block_per_state_adiabatic_jacobian_matches_oracle(mech_files, mixed_reversibility_mech, dev, idx, n):
    m, orc, ci = _handle(mech_files, mixed_reversibility_mech, idx)
    st = synth.config_states(ci, n=n, offset_seed=62)
    rho = orc.density(st.p, st.T, st.Y)
    N = orc.N
    J = m.jacobian_adiabatic(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(N, N, n)
    assert np.all(np.isfinite(J))
    Jo = orc.jacobian_adiabatic(rho, st.T, st.Y).reshape(N, N, n)
    G = orc.jacobian_adiabatic_gross(rho, st.T, st.Y).reshape(N, N, n)
    assert np.all(np.abs(J - Jo) <= TOL * G + 1e-300)


def test_block_per_state_columns_conserve_mass_and_host_arrays_match(mech_files, mixed_reversibility_mech, dev):
    m, orc, _ = _handle(mech_files, mixed_reversibility_mech, 1)
    n = 2051
    st = synth.config_states(1, n=n, offset_seed=63)
    rho = orc.density(st.p, st.T, st.Y)
    N = orc.N
    J = m.jacobian_adiabatic(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).reshape(N, N, n)
    colsum = J.sum(dim=0).abs() / (J.abs().sum(dim=0) + 1e-300)
    assert colsum.max().item() <= 1e-12
    # host arrays (staged through the library's pipeline) give the same bits
    hr, hT, hY = (np.ascontiguousarray(a) for a in (rho, st.T, st.Y))
    Jh = m.jacobian_adiabatic(hr, hT, hY)
    assert np.array_equal(Jh.reshape(N, N, n), J.cpu().numpy())
    Jd = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy()
    assert np.array_equal(m.jacobian(hr, hT, hY), Jd)


def test_block_per_state_single_and_empty(mech_files, mixed_reversibility_mech, dev):
    m, orc, _ = _handle(mech_files, mixed_reversibility_mech, 0)
    st = synth.config_states(0, n=1, offset_seed=64)
    rho = orc.density(st.p, st.T, st.Y)
    NP = orc.N + 1
    J = m.jacobian(_t(rho, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy().reshape(NP, NP, 1)
    Jo = orc.jacobian(rho, st.T, st.Y).reshape(NP, NP, 1)
    G = orc.jacobian_gross(rho, st.T, st.Y)[:, 1:]
    assert np.all(np.abs(J - Jo) <= TOL * G + 1e-300)
    e = torch.empty(0, dtype=torch.float64, device=dev)
    assert m.jacobian(e, e, torch.empty((orc.N, 0), dtype=torch.float64, device=dev)).numel() == 0


def test_block_per_state_output_alignment(mech_files, mixed_reversibility_mech, dev):
    """The dense passes write two adjacent states with one 16-byte store when the
    state count is even and J is 16-byte aligned, else one state per store: for
    both Jacobians, an output that starts 8 bytes into an allocation gives the
    bits of the aligned call, at an even and an odd state count."""
    m, orc, _ = _handle(mech_files, mixed_reversibility_mech, 1)
    NP = orc.N + 1
    for n in (64, 63):
        st = synth.config_states(1, n=n, offset_seed=65)
        rho = orc.density(st.p, st.T, st.Y)
        r, T, Y = _t(rho, dev), _t(st.T, dev), _t(st.Y, dev)
        J = m.jacobian(r, T, Y)
        buf = torch.empty(NP * NP * n + 1, dtype=torch.float64, device=dev)
        Jo = buf[1:].view(NP * NP, n)
        assert Jo.data_ptr() % 16 == 8
        m.jacobian(r, T, Y, out=Jo)
        assert torch.equal(J, Jo)
        A = m.jacobian_adiabatic(r, T, Y)
        Ao = buf[1:orc.N * orc.N * n + 1].view(orc.N * orc.N, n)
        m.jacobian_adiabatic(r, T, Y, out=Ao)
        assert torch.equal(A, Ao)
