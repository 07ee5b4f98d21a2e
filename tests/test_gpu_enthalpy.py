"""GPU parity of the enthalpy variant of the temperature inversion (Sec. A.3.1:
the Newton iteration of Eq. delta_temp with the mixture enthalpy and c_p in
place of e and c_v) against the CPU oracle, element by element on the same
seeded inputs, at sizes spanning several blocks with a ragged tail.

Tolerances: h and c_p are short FMA sums (relative error ~1e-15; bound 1e-13
relative to sum_k |Y_k h_k|, which is the natural scale under cancellation);
T as for the energy form, |dT| <= 1e-10 T.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_T = 1e-10
R = 8314.462618


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
    return {i: (B.Mechanism(paths[i]), O.Oracle(paths[i])) for i in (0, 1)}


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _abs_enthalpy_scale(orc, T, Y):
    """sum_k |Y_k h_k(T)| per state, from the oracle's species thermo."""
    out = np.zeros(T.size)
    for p in range(T.size):
        h = np.array([orc.species_thermo(k, T[p])[1] for k in range(orc.N)]) * R * T[p] / orc.W
        out[p] = np.sum(np.abs(Y[:, p] * h))
    return out + 1e-300


@pytest.mark.parametrize("idx,n", [(0, 1), (0, 4099), (1, 3001)])
def test_enthalpy_and_cp_parity(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st = synth.config_states(idx, n=n, offset_seed=11)
    h_ref, cp_ref = orc.enthalpy(st.T, st.Y, with_cp=True)
    h, cp = m.enthalpy(_t(st.T, dev), _t(st.Y, dev), with_cp=True)
    h, cp = h.cpu().numpy(), cp.cpu().numpy()
    k = min(n, 256)
    scale = _abs_enthalpy_scale(orc, st.T[:k], st.Y[:, :k])
    assert np.max(np.abs(h[:k] - h_ref[:k]) / scale) <= 1e-13
    assert np.max(np.abs(cp - cp_ref) / cp_ref) <= 1e-13


@pytest.mark.parametrize("idx,n", [(0, 4099), (1, 3001)])
def test_temperature_from_enthalpy_parity(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st = synth.config_states(idx, n=n, offset_seed=12)
    h = orc.enthalpy(st.T, st.Y)
    T_ref, it_ref, bad = orc.temperature_enthalpy(h, st.Y)
    assert bad == 0
    T, it = m.temperature_enthalpy(_t(h, dev), _t(st.Y, dev), with_iters=True)
    T, it = T.cpu().numpy(), it.cpu().numpy()
    assert np.all(it > 0) and m.nonconverged() == 0
    assert np.max(np.abs(T - T_ref) / T_ref) <= TOL_T
    assert np.max(np.abs(T - st.T) / st.T) <= TOL_T        # the round trip T -> h -> T


def test_temperature_from_enthalpy_guess_and_ragged(mechs, dev):
    """A per-state guess array is used; n not a multiple of the block; n = 0 is a no-op."""
    m, orc = mechs[0]
    st = synth.config_states(0, n=131, offset_seed=13)
    h = orc.enthalpy(st.T, st.Y)
    guess = st.T * (1.0 + 0.01 * np.sin(np.arange(st.T.size)))
    T, it = m.temperature_enthalpy(_t(h, dev), _t(st.Y, dev), guess=_t(guess, dev), with_iters=True)
    T0, it0 = m.temperature_enthalpy(_t(h, dev), _t(st.Y, dev), with_iters=True)
    assert np.max(np.abs(T.cpu().numpy() - st.T) / st.T) <= TOL_T
    assert np.max(np.abs(T0.cpu().numpy() - st.T) / st.T) <= TOL_T
    assert it.cpu().numpy().mean() < it0.cpu().numpy().mean()   # a close guess saves steps
    empty = m.temperature_enthalpy(_t(np.zeros(0), dev), _t(np.zeros((orc.N, 0)), dev))
    assert empty.numel() == 0


def test_enthalpy_minus_energy_is_p_over_rho_on_gpu(mechs, dev):
    """h - e = p/rho (Eq. eos) computed entirely by the library's kernels."""
    m, orc = mechs[1]
    st = synth.config_states(1, n=2048, offset_seed=14)
    tT, tY = _t(st.T, dev), _t(st.Y, dev)
    rho = m.density(_t(st.p, dev), tT, tY)
    h = m.enthalpy(tT, tY)
    e = m.internal_energy(tT, tY)
    lhs = (h - e).cpu().numpy()
    assert np.allclose(lhs, st.p / rho.cpu().numpy(), rtol=1e-12, atol=0)
