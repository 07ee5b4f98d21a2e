"""GPU parity of the forward path against the CPU oracle (element by element on
the same seeded inputs), at oracle-sized cases spanning several blocks with a
ragged tail, and at the full 2^22-point workload (sampled points plus
properties that hold at any size).

Tolerances (the FP64 kernels reorder sums and use table-driven exp/log of
<= 2 ulp, so relative errors stay ~1e-14 per term; the bounds leave margin):
  T:      |dT| <= 1e-10 T
  omega:  |d omega_k| <= 1e-11 G_k, G_k = sum_j |nu_kj| (|Rf_j| + |Rr_j|) (oracle)
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_T = 1e-10
TOL_W = 1e-11


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


def _inputs(idx, n, orc, seed_offset=0):
    st = synth.config_states(idx, n=n, offset_seed=seed_offset)
    rho = orc.density(st.p, st.T, st.Y)
    e = orc.internal_energy(st.T, st.Y)
    return st, rho, e


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


# --- device math ----------------------------------------------------------------

def test_device_math_accuracy(mechs, dev):
    m = mechs[0][0]
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-700, 700, 200000), np.linspace(-1, 1, 20001), [0.0, 1e-300, -1e-300]])
    y = m.math_eval(0, _t(x, dev)).cpu().numpy()
    assert np.max(np.abs(y - np.exp(x)) / np.exp(x)) <= 4.5e-16          # ~2 ulp
    x = np.exp(rng.uniform(-700, 700, 200000))
    y = m.math_eval(1, _t(x, dev)).cpu().numpy()
    assert np.max(np.abs(y - np.log(x)) / np.maximum(1.0, np.abs(np.log(x)))) <= 4.5e-16
    y = m.math_eval(2, _t(x, dev)).cpu().numpy()
    assert np.max(np.abs(y * x - 1.0)) <= 4.5e-16
    # out-of-range arguments take the library path, not garbage
    xe = np.array([-800.0, 710.0, -745.0])
    ye = m.math_eval(0, _t(xe, dev)).cpu().numpy()
    assert ye[0] == 0.0 and np.isinf(ye[1]) and ye[2] == pytest.approx(np.exp(-745.0), rel=1e-3)
    yl = m.math_eval(1, _t(np.array([0.0, -1.0, 1e-310]), dev)).cpu().numpy()
    assert np.isneginf(yl[0]) and np.isnan(yl[1]) and yl[2] == pytest.approx(np.log(1e-310), rel=1e-12)


# --- mixture relations ---------------------------------------------------------------

@pytest.mark.parametrize("idx", [0, 1])
def test_density_and_energy_parity(mechs, dev, idx):
    m, orc = mechs[idx]
    st, rho, e = _inputs(idx, 3000, orc)
    g_rho = m.density(_t(st.p, dev), _t(st.T, dev), _t(st.Y, dev)).cpu().numpy()
    assert np.max(np.abs(g_rho - rho) / rho) <= 1e-14
    g_e, g_cv = m.internal_energy(_t(st.T, dev), _t(st.Y, dev), with_cv=True)
    _, cv = orc.internal_energy(st.T, st.Y, with_cv=True)
    scale = cv * st.T
    assert np.max(np.abs(g_e.cpu().numpy() - e) / scale) <= 1e-13
    assert np.max(np.abs(g_cv.cpu().numpy() - cv) / cv) <= 1e-13


# --- temperature ---------------------------------------------------------------

@pytest.mark.parametrize("idx,n", [(0, 4096), (0, 1), (0, 257), (1, 1500)])
def test_temperature_parity(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho, e = _inputs(idx, n, orc)
    T, it = m.temperature(_t(e, dev), _t(st.Y, dev), with_iters=True)
    T, it = T.cpu().numpy(), it.cpu().numpy()
    oT, oit, bad = orc.temperature(e, st.Y)
    assert bad == 0 and m.nonconverged() == 0
    assert np.all(it > 0)
    assert np.max(np.abs(T - oT) / oT) <= TOL_T
    # both recover the generating temperature (the problem has a unique root)
    assert np.max(np.abs(T - st.T) / st.T) <= 1e-12


def test_temperature_with_guess_array_and_fp64_newton(mechs, dev, mech_files):
    from paper_2503_24286_gb300 import binding as B
    m, orc = mechs[0]
    st, rho, e = _inputs(0, 2000, orc, seed_offset=3)
    guess = st.T * (1.0 + 0.05 * np.sin(np.arange(st.T.size)))
    T, it = m.temperature(_t(e, dev), _t(st.Y, dev), guess=_t(guess, dev), with_iters=True)
    oT, _, _ = orc.temperature(e, st.Y, guess=guess)
    assert np.max(np.abs(T.cpu().numpy() - oT) / oT) <= TOL_T
    m64 = B.Mechanism(mech_files[0][0], "newton=fp64")
    T2, it2 = m64.temperature(_t(e, dev), _t(st.Y, dev), with_iters=True)
    oT2, oit2, _ = orc.temperature(e, st.Y)
    assert np.max(np.abs(T2.cpu().numpy() - oT2) / oT2) <= TOL_T
    # the FP64 variant follows the paper's iteration from 1200 K: same step counts
    assert np.mean(np.abs(it2.cpu().numpy() - oit2)) <= 0.05


def test_temperature_nonconvergence_is_reported(mechs, dev, mech_files):
    from paper_2503_24286_gb300 import binding as B
    m, orc = mechs[0]
    st, rho, e = _inputs(0, 64, orc)
    e_bad = e.copy()
    e_bad[3] = np.nan
    e_bad[7] = 1e12          # no temperature below the 5000 K clamp has this energy
    T, it = m.temperature(_t(e_bad, dev), _t(st.Y, dev), with_iters=True)
    it = it.cpu().numpy()
    assert it[3] == -1 and it[7] == -1
    assert np.all(np.delete(it, [3, 7]) > 0)
    assert m.nonconverged() == 2
    assert m.nonconverged() == 0          # counter resets
    mc = B.Mechanism(mech_files[0][0], "checked=1")
    with pytest.raises(B.PyroError) as ei:
        mc.temperature(_t(e_bad, dev), _t(st.Y, dev))
    assert ei.value.code == B.PYRO_ENOCONV


# --- net production rates -----------------------------------------------------------

@pytest.mark.parametrize("idx,n", [(0, 4096), (0, 1), (0, 1000), (1, 1029)])
def test_omega_isothermal_parity(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho, e = _inputs(idx, n, orc)
    w = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), T=_t(st.T, dev)).cpu().numpy()
    ow, G = orc.net_production_rates(rho, st.T, st.Y, with_gross=True)
    assert np.all(np.isfinite(w))
    assert np.all(np.abs(w - ow) <= TOL_W * G + 1e-300)


@pytest.mark.parametrize("idx,n", [(0, 4096), (1, 777)])
def test_omega_energy_parity(mechs, dev, idx, n):
    m, orc = mechs[idx]
    st, rho, e = _inputs(idx, n, orc, seed_offset=1)
    w, T = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
    w, T = w.cpu().numpy(), T.cpu().numpy()
    oT, _, bad = orc.temperature(e, st.Y)
    ow, G = orc.net_production_rates(rho, oT, st.Y, with_gross=True)
    assert bad == 0 and m.nonconverged() == 0
    assert np.max(np.abs(T - oT) / oT) <= TOL_T
    assert np.all(np.abs(w - ow) <= TOL_W * G + 1e-300)


def test_omega_edge_states(mechs, dev):
    """Species absent (Y_k = 0), a single-species state, T at the NASA range switch
    and at the ends of the sampled range."""
    m, orc = mechs[1]
    N = orc.N
    st, rho, e = _inputs(1, 64, orc, seed_offset=9)
    Y = st.Y.copy()
    Y[::3, 0:8] = 0.0
    Y[:, 0:8] /= Y[:, 0:8].sum(axis=0)
    Y[:, 8] = 0.0
    Y[5, 8] = 1.0
    T = st.T.copy()
    T[9:14] = [1000.0, np.nextafter(1000.0, 0.0), np.nextafter(1000.0, 2000.0), 300.0, 2800.0]
    rho = orc.density(st.p, T, Y)
    w = m.net_production_rates(_t(rho, dev), _t(Y, dev), T=_t(T, dev)).cpu().numpy()
    ow, G = orc.net_production_rates(rho, T, Y, with_gross=True)
    assert np.all(np.isfinite(w))
    assert np.all(np.abs(w - ow) <= TOL_W * G + 1e-300)


def test_host_pointer_path_matches(mechs, dev):
    """numpy (host) arrays are staged by the library and give the same bits."""
    m, orc = mechs[0]
    st, rho, e = _inputs(0, 999, orc)
    wh, Th = m.net_production_rates(rho, np.ascontiguousarray(st.Y), e=e)
    wd, Td = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
    assert np.array_equal(wh, wd.cpu().numpy()) and np.array_equal(Th, Td.cpu().numpy())


def test_host_pointer_pipeline_chunks(mechs, dev):
    """Host arrays larger than one staging chunk (65536 points) go through the
    chunked copy/kernel pipeline: chunks ramping from 8192 points up to 65536 and
    back down, over the three staging slots, with a ragged chunk, for [N][n] and [n]
    arrays, FP64 and int32 outputs, with the chunks' kernels overlapping (forward,
    temperature) or chained (Jacobian); every output equals the device-pointer
    call bit for bit."""
    m, orc = mechs[0]
    n = 5 * 65536 + 37
    cfg = synth.CONFIGS[0]
    T0, p, Y = synth.generate_states_torch(10, n, cfg["T"], cfg["p_atm"], 4242, dev)
    rho = m.density(p, T0, Y)
    e = m.internal_energy(T0, Y)
    wd, Td = m.net_production_rates(rho, Y, e=e)
    Tt, itd = m.temperature(e, Y, with_iters=True)
    hr, hY, he = (np.ascontiguousarray(x.cpu().numpy()) for x in (rho, Y, e))
    wh, Th = m.net_production_rates(hr, hY, e=he)
    Th2, ith = m.temperature(he, hY, with_iters=True)
    assert np.array_equal(wh, wd.cpu().numpy()) and np.array_equal(Th, Td.cpu().numpy())
    assert np.array_equal(Th2, Tt.cpu().numpy()) and np.array_equal(ith, itd.cpu().numpy())
    # Jacobian ([(N+1)^2][n] output; its kernels share per-block scratch, so the
    # chunks' kernels run one after another) over ramped chunks and a ragged one
    nj = 3 * 65536 + 5
    Jd = m.jacobian(rho[:nj].contiguous(), Td[:nj].contiguous(), Y[:, :nj].contiguous())
    Jh = m.jacobian(hr[:nj].copy(), np.ascontiguousarray(Th[:nj]), np.ascontiguousarray(hY[:, :nj]))
    assert np.array_equal(Jh, Jd.cpu().numpy())


def test_mixed_host_device_rejected(mechs, dev):
    from paper_2503_24286_gb300 import binding as B
    m, orc = mechs[0]
    st, rho, e = _inputs(0, 16, orc)
    with pytest.raises(B.PyroError) as ei:
        m.net_production_rates(_t(rho, dev), np.ascontiguousarray(st.Y), T=_t(st.T, dev))
    assert ei.value.code == B.PYRO_EINVAL


def test_full_size_workload_sampled(mechs, dev):
    """The bench workload (53 species, 325 reactions, 2^22 points, energy input) in
    the bench's launch configuration; sampled points against the oracle and the
    generating temperature at every point."""
    m, orc = mechs[1]
    n = synth.CONFIGS[1]["n_points"]
    T0, p, Y = synth.generate_states_torch(53, n, synth.CONFIGS[1]["T"], synth.CONFIGS[1]["p_atm"],
                                           synth.STATE_SEED_BASE + 1, dev)
    rho = m.density(p, T0, Y)
    e = m.internal_energy(T0, Y)
    w, T = m.net_production_rates(rho, Y, e=e)
    torch.cuda.synchronize()
    assert m.nonconverged() == 0
    assert torch.isfinite(w).all().item()
    assert (torch.abs(T - T0) / T0).max().item() <= 1e-12
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, 1, n - 2, n - 1], rng.integers(0, n, 400)]))
    ii = torch.tensor(idx, device=dev)
    Ys = Y[:, ii].cpu().numpy()
    es, rhos = e[ii].cpu().numpy(), rho[ii].cpu().numpy()
    oT, _, bad = orc.temperature(es, Ys)
    ow, G = orc.net_production_rates(rhos, oT, Ys, with_gross=True)
    assert bad == 0
    assert np.max(np.abs(T[ii].cpu().numpy() - oT) / oT) <= TOL_T
    assert np.all(np.abs(w[:, ii].cpu().numpy() - ow) <= TOL_W * G + 1e-300)


@pytest.mark.parametrize("idx", [0, 1, 7, "7-mixed"])
def test_warp_variant_parity(mechs, dev, mech_files, mixed_reversibility_mech, idx):
    """One warp per state (the emitted warp-per-state kernel, lanes splitting the
    species and the reactions) gives the oracle's results as well, including the
    SRI and PLOG reactions of the pressure-dependent variant and, with every third
    reaction irreversible, reactions of both directions in one class."""
    from paper_2503_24286_gb300 import binding as B
    path = mixed_reversibility_mech if idx == "7-mixed" else mech_files[0][idx]
    orc = mechs[idx][1] if idx in mechs else O.Oracle(path)
    m = B.Mechanism(path, "variant=warp")
    idx = 7 if idx == "7-mixed" else idx
    assert m.stat("variant_warp") == 1
    st, rho, e = _inputs(idx, 777, orc, seed_offset=11)
    w = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), T=_t(st.T, dev)).cpu().numpy()
    ow, G = orc.net_production_rates(rho, st.T, st.Y, with_gross=True)
    assert np.all(np.abs(w - ow) <= TOL_W * G + 1e-300)
    w2, T2 = m.net_production_rates(_t(rho, dev), _t(st.Y, dev), e=_t(e, dev))
    oT, _, _ = orc.temperature(e, st.Y)
    assert m.nonconverged() == 0
    assert np.max(np.abs(T2.cpu().numpy() - oT) / oT) <= TOL_T
    ow2, G2 = orc.net_production_rates(rho, oT, st.Y, with_gross=True)
    assert np.all(np.abs(w2.cpu().numpy() - ow2) <= TOL_W * G2 + 1e-300)
