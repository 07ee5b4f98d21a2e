"""GPU parity of the mixture-averaged transport properties (Sec. A.2) against the
CPU oracle, element by element on the same seeded inputs, at sizes spanning
several blocks with a ragged tail, for the 10-, 53- and 160-species mechanisms,
and at the 2^20-state benchmark size on sampled states.

Tolerances (relative).  The fits are quartics in ln T over [250, 3600] K whose
alternating coefficients cancel: by up to ~3e2 (viscosity bracket), ~8e2
(conductivity) and ~1e4 (binary diffusivity) in sum_m a_m ln^m T.  Each side's
rounding error is that factor times a few ulp, so mu and kappa agree to
~1e-13 and D_km to ~5e-12; the bounds are 1e-12 (mu, kappa) and 2e-11 (D_km).
The Wilke sums and the diffusion sums add positive terms only.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MU = 1e-12
TOL_K = 1e-12
TOL_D = 2e-11


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
    for i in (0, 1, 4):
        m = B.Mechanism(paths[i])
        m.prepare("transport")
        out[i] = (m, O.Oracle(paths[i]))
    return out


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _rel(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


@pytest.mark.parametrize("idx,n", [(0, 1), (0, 4099), (1, 1001), (4, 257)])
def test_transport_matches_oracle(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st = synth.config_states(idx, n=n, offset_seed=31)
    mu, ka, Dm = (x.cpu().numpy() for x in m.transport(_t(st.T, dev), _t(st.Y, dev)))
    omu, oka, oDm = orc.transport(st.T, st.Y)
    assert np.all(np.isfinite(mu)) and np.all(np.isfinite(ka)) and np.all(np.isfinite(Dm))
    assert _rel(mu, omu) <= TOL_MU
    assert _rel(ka, oka) <= TOL_K
    assert _rel(Dm, oDm) <= TOL_D


def test_transport_optional_outputs_host_arrays_and_errors(mechs, dev, tmp_path):
    m, orc = mechs[1]
    st = synth.config_states(1, n=700, offset_seed=32)
    T, Y = _t(st.T, dev), _t(st.Y, dev)
    mu, ka, Dm = m.transport(T, Y)
    mu1, k1, d1 = m.transport(T, Y, kappa=False, diffusivities=False)
    assert k1 is None and d1 is None and torch.equal(mu1, mu)
    _, k2, d2 = m.transport(T, Y, mu=False)
    assert torch.equal(k2, ka) and torch.equal(d2, Dm)
    # host arrays give the same bits
    hm, hk, hd = m.transport(st.T, st.Y)
    assert np.array_equal(hm, mu.cpu().numpy()) and np.array_equal(hd, Dm.cpu().numpy())
    # n = 0 is a no-op
    z = m.transport(_t(np.zeros(0), dev), _t(np.zeros((orc.N, 0)), dev))
    assert z[0].numel() == 0
    # a mechanism without a transport section is rejected
    from paper_2503_24286_gb300 import binding as B
    from tests import handmech
    p = handmech.write(handmech.abcd_mechanism(), str(tmp_path), "abcd.txt")
    mb = B.Mechanism(p)
    with pytest.raises(B.PyroError) as ei:
        mb.transport(_t(np.full(4, 1000.0), dev), _t(np.full((4, 4), 0.25), dev))
    assert ei.value.code == B.PYRO_EMECH


def test_transport_full_size_sampled(mechs, dev):
    """2^20 states of the 53-species workload: all finite and positive, sampled
    states against the oracle."""
    m, orc = mechs[1]
    n = 2 ** 20
    cfg = synth.CONFIGS[1]
    T, p, Y = synth.generate_states_torch(53, n, cfg["T"], cfg["p_atm"], synth.STATE_SEED_BASE + 1 + 17, dev)
    mu, ka, Dm = m.transport(T, Y)
    assert (mu > 0).all().item() and (ka > 0).all().item() and (Dm > 0).all().item()
    assert torch.isfinite(Dm).all().item()
    idx = np.array([0, 1, 4242, n // 2, n - 1])
    ii = torch.tensor(idx, device=dev)
    omu, oka, oDm = orc.transport(T[ii].cpu().numpy(), Y[:, ii].cpu().numpy())
    assert _rel(mu[ii].cpu().numpy(), omu) <= TOL_MU
    assert _rel(ka[ii].cpu().numpy(), oka) <= TOL_K
    assert _rel(Dm[:, ii].cpu().numpy(), oDm) <= TOL_D
