"""The entry point that allocates no device memory, checked against the regular one.

pyro_net_production_rates_noalloc serves callers that cannot call cudaMalloc
while they evaluate the chemistry (a solver whose memory pool already holds the
whole device, or a loop that must not take cudaMalloc's device-wide
synchronisation).  It stages the arrays through one fixed scratch array held by
the library, so this test calls it twice in a row -- the second call finds the
first call's contents in the scratch -- and compares both with
pyro_net_production_rates on the same inputs, within the parity tolerance of the
forward tests.  It also checks that a call larger than the scratch is refused,
that a call leaves the device's free memory unchanged (nothing allocated), and
that it runs the handle's own kernel for the warp-per-state variant and for the
160-species mechanism (species arrays in the handle's global scratch).

This file is collected last so that a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_W = 1e-11


@pytest.fixture(scope="module")
def setup(mech_files):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    paths, _ = mech_files
    return B, B.Mechanism(paths[1]), O.Oracle(paths[1])


def _case(orc, n, seed):
    st = synth.config_states(1, n=n, offset_seed=seed)
    rho = orc.density(st.p, st.T, st.Y)
    e = orc.internal_energy(st.T, st.Y)
    return st, rho, e


def test_noalloc_matches_regular_entry_point_twice(setup):
    B, mech, orc = setup
    dev = torch.device("cuda:0")
    for call, (n, seed) in enumerate([(3001, 41), (1777, 42)]):
        st, rho, e = _case(orc, n, seed)
        # regular entry point on device arrays
        w_ref, T_ref = mech.net_production_rates(torch.tensor(rho, device=dev), torch.tensor(st.Y, device=dev),
                                                 e=torch.tensor(e, device=dev))
        w_ref, T_ref = w_ref.cpu().numpy(), T_ref.cpu().numpy()
        # no-allocation entry point on host arrays (energy input), through the C ABI
        w, T = mech.net_production_rates_noalloc(rho, np.ascontiguousarray(st.Y), e=e)
        _, G = orc.net_production_rates(rho, T_ref, st.Y, with_gross=True)
        assert np.max(np.abs(T - T_ref) / T_ref) <= 1e-10, call
        assert np.all(np.abs(w - w_ref) <= TOL_W * G + 1e-300), call
        # temperature input, device arrays
        tT = torch.tensor(st.T, device=dev)
        w2 = mech.net_production_rates_noalloc(torch.tensor(rho, device=dev), torch.tensor(st.Y, device=dev), T=tT)
        w2_ref = mech.net_production_rates(torch.tensor(rho, device=dev), torch.tensor(st.Y, device=dev), T=tT)
        _, G2 = orc.net_production_rates(rho, st.T, st.Y, with_gross=True)
        assert np.all(np.abs(w2.cpu().numpy() - w2_ref.cpu().numpy()) <= TOL_W * G2 + 1e-300), call


def test_noalloc_rejects_calls_beyond_the_scratch(setup):
    B, mech, orc = setup
    n = 40000                      # 53 species: 8 * (2*53 + 3) B/state -> ~38 000 states fit
    rho = np.ones(n)
    Y = np.full((53, n), 1.0 / 53)
    with pytest.raises(B.PyroError) as ei:
        mech.net_production_rates_noalloc(rho, Y, T=np.full(n, 1000.0))
    assert ei.value.code == B.PYRO_EINVAL
    assert "scratch" in str(ei.value)


def test_noalloc_allocates_no_device_memory(setup):
    """After a warm-up call, a call on host arrays leaves the driver's free device
    memory exactly as it was."""
    B, mech, orc = setup
    st, rho, e = _case(orc, 2048, 43)
    Y = np.ascontiguousarray(st.Y)
    mech.net_production_rates_noalloc(rho, Y, e=e)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    w, T = mech.net_production_rates_noalloc(rho, Y, e=e)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.all(np.isfinite(w))


@pytest.mark.parametrize("idx,opts", [(1, "variant=warp"), (4, None)])
def test_noalloc_runs_the_handles_kernel(mech_files, idx, opts):
    """The warp-per-state handle and the 160-species handle (store=global): two calls
    in a row against the regular entry point on the same handle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    paths, _ = mech_files
    m = B.Mechanism(paths[idx], opts)
    orc = O.Oracle(paths[idx])
    if idx == 4:
        assert m.stat("omega_store_global") == 1
    else:
        assert m.stat("variant_warp") == 1
    dev = torch.device("cuda:0")
    for call, (n, seed) in enumerate([(517, 44), (301, 45)]):
        st = synth.config_states(idx, n=n, offset_seed=seed)
        rho = orc.density(st.p, st.T, st.Y)
        e = orc.internal_energy(st.T, st.Y)
        w_ref, T_ref = m.net_production_rates(torch.tensor(rho, device=dev), torch.tensor(st.Y, device=dev),
                                              e=torch.tensor(e, device=dev))
        w, T = m.net_production_rates_noalloc(rho, np.ascontiguousarray(st.Y), e=e)
        T_ref = T_ref.cpu().numpy()
        _, G = orc.net_production_rates(rho, T_ref, st.Y, with_gross=True)
        assert np.max(np.abs(T - T_ref) / T_ref) <= 1e-10, call
        assert np.all(np.abs(w - w_ref.cpu().numpy()) <= TOL_W * G + 1e-300), call
