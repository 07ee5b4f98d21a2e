"""Pins of the oracle's mixture-averaged transport (Sec. A.2: species fits,
Eq. mixavg_viscosity with Wilke's Phi, Eq. mixavg_conductivity,
Eq. diff_mix_rule) against what the physics and the algebra fix, independently
of the oracle's own formulas:

* the species fits reproduce the generator's Chapman-Enskog-type model curves
  they were fitted to (pins the squared bracket, the sqrt(T) factor, ln T);
* Phi_kk = 1 and the reciprocity Phi_jk = Phi_kj (mu_j/mu_k)(W_k/W_j) of
  Wilke's rule (pins the operand order and both exponents of W);
* pure-species limits; a mixture of identical isomers behaves as one species;
* in a binary mixture the mixture-averaged flux of Eq. mixavg_flux is exactly
  Fick's law with the binary diffusivity, -rho D_12 dY_1/dx, and the two
  fluxes cancel (pins the (W - X_k W_k)/W factor and the 1/D_kj sum);
* the long-double envelope of the double oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth
from tests import handmech


@pytest.fixture(scope="module")
def orc(mech_files):
    paths, _ = mech_files
    return {i: O.Oracle(paths[i]) for i in (0, 1)}


def _model(idx):
    mech = synth.config_mechanism(idx)
    return mech, synth.transport_model(mech, synth.MECH_SEED_BASE + synth.TRANSPORT_SEED_OFFSET
                                       + synth.CONFIGS[idx]["mech"])


@pytest.mark.parametrize("idx", [0, 1])
def test_species_fits_reproduce_the_generating_model(orc, idx):
    o = orc[idx]
    assert o.has_transport
    mech, mdl = _model(idx)
    T = np.linspace(300.0, 3500.0, 23)
    mu_ref, k_ref, D_ref = mdl.viscosity(T), mdl.conductivity(T), mdl.diffusivity(T)
    mu = np.array([[o.species_transport(k, t)[0] for t in T] for k in range(o.N)])
    ka = np.array([[o.species_transport(k, t)[1] for t in T] for k in range(o.N)])
    assert np.max(np.abs(mu / mu_ref - 1)) < 1e-2
    assert np.max(np.abs(ka / k_ref - 1)) < 1e-2
    rng = np.random.default_rng(0)
    for _ in range(40):
        k, j = rng.choice(o.N, size=2, replace=False)
        D = np.array([o.binary_diffusivity(k, j, t) for t in T])
        assert np.max(np.abs(D / D_ref[k, j] - 1)) < 4e-2
        assert np.array_equal(D, [o.binary_diffusivity(j, k, t) for t in T])   # symmetric


@pytest.mark.parametrize("T", [300.0, 999.0, 1800.0, 3200.0])
def test_wilke_phi_diagonal_and_reciprocity(orc, T):
    o = orc[1]
    Phi = o.wilke_phi(T)
    mu = np.array([o.species_transport(k, T)[0] for k in range(o.N)])
    W = o.W
    assert np.allclose(np.diag(Phi), 1.0, rtol=1e-15, atol=0)
    # Phi_jk = Phi_kj (mu_j / mu_k) (W_k / W_j): with k the row index, Phi.T[k, j] = Phi_jk
    lhs = Phi.T
    rhs = Phi * (mu[None, :] / mu[:, None]) * (W[:, None] / W[None, :])
    assert np.max(np.abs(lhs / rhs - 1)) < 1e-13


def test_pure_species_limits(orc):
    o = orc[0]
    T = np.array([400.0, 1200.0, 2600.0])
    for k in range(o.N):
        Y = np.zeros((o.N, T.size))
        Y[k] = 1.0
        mu, ka, Dm = o.transport(T, Y)
        mk = np.array([o.species_transport(k, t) for t in T])
        assert np.allclose(mu, mk[:, 0], rtol=1e-14, atol=0)
        assert np.allclose(ka, mk[:, 1], rtol=1e-14, atol=0)
        # every other species diffuses into pure k with the binary coefficient D_jk
        for j in range(o.N):
            if j != k:
                Djk = np.array([o.binary_diffusivity(j, k, t) for t in T])
                assert np.allclose(Dm[j], Djk, rtol=1e-14, atol=0)


def _isomers(tmp_path):
    els = [("C", synth.ATOMIC_WEIGHTS["C"]), ("O", synth.ATOMIC_WEIGHTS["O"])]
    sp = [handmech.const_cp_species("A", {"C": 1, "O": 1}, 3.5, -1.3e4, 20.0),
          handmech.const_cp_species("B", {"C": 1, "O": 1}, 3.5, -1.3e4, 20.0)]
    r = synth.Reaction("arrhenius", [(0, 1)], [(1, 1)], 1e8, 0.0, 1000.0)
    mech = synth.Mechanism("iso", els, sp, [r])
    b = np.array([2.0e-3, 1.0e-4, -2.0e-5, 1.0e-6, 0.0])
    c = np.array([1.0e-3, 5.0e-4, -1.0e-5, 0.0, 0.0])
    a = np.array([-1.0e-5, 4.0e-6, 0.0, 0.0, 0.0])
    diff = np.zeros((2, 2, 5))
    diff[0, 1] = diff[1, 0] = a
    mech.transport = synth.Transport(np.stack([b, b]), np.stack([c, c]), diff)
    return O.Oracle(handmech.write(mech, str(tmp_path), "iso.txt"))


def test_identical_isomers_mix_as_one_species(tmp_path):
    o = _isomers(tmp_path)
    rng = np.random.default_rng(1)
    T = rng.uniform(300, 3000, 50)
    y1 = rng.uniform(0.01, 0.99, 50)
    Y = np.stack([y1, 1 - y1])
    mu, ka, Dm = o.transport(T, Y)
    mk = np.array([o.species_transport(0, t) for t in T])
    D12 = np.array([o.binary_diffusivity(0, 1, t) for t in T])
    assert np.allclose(mu, mk[:, 0], rtol=1e-14, atol=0)
    assert np.allclose(ka, mk[:, 1], rtol=1e-14, atol=0)
    assert np.allclose(Dm, D12[None], rtol=1e-14, atol=0)


def test_binary_mixture_flux_is_ficks_law(tmp_path):
    """H2 / N2: phi*_1 = -rho D_1m (W_1/W) dX_1/dx equals -rho D_12 dY_1/dx for any
    gradient (dX_1/dY_1 by central differences of the mole-fraction map, computed
    here from the molecular weights alone), and phi*_1 + phi*_2 = 0."""
    els = [("H", synth.ATOMIC_WEIGHTS["H"]), ("N", synth.ATOMIC_WEIGHTS["N"])]
    sp = [handmech.const_cp_species("H2", {"H": 2}, 3.5, 0.0, 15.0),
          handmech.const_cp_species("N2", {"N": 2}, 3.5, 0.0, 23.0)]
    mech = synth.Mechanism("h2n2", els, sp, [])
    mech.transport = synth.generate_transport(mech, 7)
    o = O.Oracle(handmech.write(mech, str(tmp_path), "h2n2.txt"))
    W1, W2 = o.W
    rng = np.random.default_rng(2)
    T = rng.uniform(300, 3000, 40)
    y1 = rng.uniform(0.05, 0.95, 40)
    _, _, Dm = o.transport(T, np.stack([y1, 1 - y1]))
    D12 = np.array([o.binary_diffusivity(0, 1, t) for t in T])

    def x1(y):
        return (y / W1) / (y / W1 + (1 - y) / W2)
    h = 1e-6
    dx1 = (x1(y1 + h) - x1(y1 - h)) / (2 * h)
    Wmix = 1.0 / (y1 / W1 + (1 - y1) / W2)
    assert np.allclose(Dm[0] * (W1 / Wmix) * dx1, D12, rtol=1e-8, atol=0)
    assert np.allclose(Dm[1] * (W2 / Wmix) * dx1, D12, rtol=1e-8, atol=0)   # dX_2/dY_2 = dX_1/dY_1
    assert np.allclose(Dm[0] * W1, Dm[1] * W2, rtol=1e-14, atol=0)           # fluxes cancel


def test_mixture_values_bounded_and_long_double_envelope(orc):
    o = orc[1]
    st = synth.config_states(1, n=64, offset_seed=9)
    mu, ka, Dm = o.transport(st.T, st.Y)
    mu_l, ka_l, Dm_l = o.transport(st.T, st.Y, long_double=True)
    assert np.max(np.abs(mu / mu_l - 1)) < 1e-13
    assert np.max(np.abs(ka / ka_l - 1)) < 1e-13
    # the binary-diffusivity fits cancel by up to ~1e4 in sum_m a_m ln^m T (alternating
    # coefficients of a quartic over [250, 3600] K), so their rounding error is ~1e4 ulp
    assert np.max(np.abs(Dm / Dm_l - 1)) < 5e-12
    for p in range(0, 64, 8):
        sk = np.array([o.species_transport(k, st.T[p]) for k in range(o.N)])
        assert sk[:, 1].min() <= ka[p] <= sk[:, 1].max()
        assert np.all(Dm[:, p] > 0) and np.isfinite(Dm[:, p]).all()


def test_transport_section_round_trip(tmp_path):
    mech = synth.config_mechanism(0)
    p = handmech.write(mech, str(tmp_path), "m0.txt")
    back = synth.read_mechanism(p)
    assert np.array_equal(back.transport.visc, mech.transport.visc)
    assert np.array_equal(back.transport.cond, mech.transport.cond)
    assert np.array_equal(back.transport.diff, mech.transport.diff)
