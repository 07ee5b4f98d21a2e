"""Learned initial guess: the BF16 tensor-core network and the hand-written
training kernels against the CPU oracle's FP64 model definition (same bf16
rounding points), then training on states the plain method generates and the
Newton-iteration gain it gives at unchanged accuracy.

Tolerances: the GPU accumulates in FP32 while the oracle uses FP64, so a hidden
activation can land on the other side of a bf16 rounding boundary (one bf16 ulp
= 2^-8 relative); the network output then moves by ~1e-3 in normalised units.
The test allows 1e-2 at any point and 1e-5 at the median.  Gradients: the same
effect, relative to the largest gradient entry: 2e-3.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 64


def bf16(x):
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def mech1(mech_files, dev):
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    return B.Mechanism(mech_files[0][1]), O.Oracle(mech_files[0][1]), mech_files[0][1]


def _t(a, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def _random_params(D, seed):
    rng = np.random.default_rng(seed)
    P = O.mlp_n_params(D, H)
    p = np.zeros(P)
    W1 = bf16(rng.uniform(-1, 1, H * D) / np.sqrt(D))
    b1 = rng.uniform(-0.5, 0.5, H).astype(np.float32).astype(np.float64)
    W2 = bf16(rng.uniform(-1, 1, H * H) / np.sqrt(H))
    b2 = rng.uniform(-0.5, 0.5, H).astype(np.float32).astype(np.float64)
    w3 = bf16(rng.uniform(-1, 1, H) / np.sqrt(H))
    b3 = np.float32(0.1)
    p[:] = np.concatenate([W1, b1, W2, b2, w3, [b3]])
    return p


def _trunc32(x):
    """double -> float32 by truncating the mantissa, tiny values to zero (feature definition)."""
    u = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64) & np.uint64(0xFFFFFFFFE0000000)
    f = u.view(np.float64).astype(np.float32)          # exact: no bits left below float precision
    f[np.abs(f) < np.float32(1.1754944e-38)] = 0.0
    return f


def _features(e, Y, norm):
    e_mean = np.float32(norm[0])
    e_inv = np.float32(1.0) / np.float32(norm[1])
    x0 = ((e - np.float64(e_mean)) * np.float64(e_inv)).astype(np.float32).astype(np.float64)
    N = Y.shape[0]
    xy = (_trunc32(Y) * np.float32(N)).astype(np.float64)
    return np.concatenate([x0[:, None], xy.T], axis=1)          # [n, D]


def _states(orc, n, seed):
    st = synth.config_states(3, n=n, offset_seed=seed)
    e = orc.internal_energy(st.T, st.Y)
    return st, e


def test_network_matches_oracle_model(mech1, dev):
    m, orc, _ = mech1
    D = orc.N + 1
    p = _random_params(D, 1)
    st, e = _states(orc, 3000, 7)
    norm = np.array([e.mean(), e.std(), 1550.0, 720.0])
    m.mlp_set_params(p, norm)
    y, Tg = m.mlp_guess(_t(e, dev), _t(st.Y, dev))
    y, Tg = y.cpu().numpy(), Tg.cpu().numpy()
    yo = O.mlp_forward(D, H, p, _features(e, st.Y, norm))
    err = np.abs(y - yo)
    assert np.max(err) <= 1e-2 and np.median(err) <= 1e-5
    Tref = np.clip(np.float32(norm[2]) + np.float32(norm[3]) * y.astype(np.float32), 200.0, 3500.0)
    assert np.allclose(Tg, Tref, rtol=1e-6)


def test_training_gradient_matches_oracle(mech1, dev):
    m, orc, _ = mech1
    D = orc.N + 1
    p = _random_params(D, 2)
    st, e = _states(orc, 256, 8)
    norm = np.array([e.mean(), e.std(), st.T.mean(), st.T.std()])
    m.mlp_set_params(p, norm)
    loss, g = m.mlp_grad(_t(e, dev), _t(st.Y, dev), _t(st.T, dev))
    t = ((st.T - np.float32(norm[2])) / np.float32(norm[3]))
    lo, go = O.mlp_loss_grad(D, H, p, _features(e, st.Y, norm), t)
    assert loss == pytest.approx(lo, rel=2e-3)
    assert np.max(np.abs(g - go)) <= 2e-3 * np.max(np.abs(go))


def test_training_and_newton_gain(mech1, dev, mech_files, tmp_path):
    """Train on states the plain method generates; the learned guess must leave T
    at oracle accuracy while cutting the Newton steps of both solve variants."""
    from paper_2503_24286_gb300 import binding as B
    m, orc, path = mech1
    n_train = 2 ** 19
    cfg = synth.CONFIGS[3]
    T, p, Y = synth.generate_states_torch(53, n_train, cfg["T"], cfg["p_atm"], 777, dev)
    loss = m.mlp_train(T, Y, "epochs=6;batch=1024;lr=1e-2;seed=3")
    assert loss < 2e-3, loss
    st, e = _states(orc, 4096, 9)               # held out
    te, tY = _t(e, dev), _t(st.Y, dev)
    T0, it0 = m.temperature(te, tY, with_iters=True)
    T1, it1 = m.temperature(te, tY, learned=True, with_iters=True)
    oT, _, bad = orc.temperature(e, st.Y)
    T1, it1, it0 = T1.cpu().numpy(), it1.cpu().numpy(), it0.cpu().numpy()
    assert bad == 0 and m.nonconverged() == 0
    assert np.max(np.abs(T1 - oT) / oT) <= 1e-10
    assert np.all(it1 > 0)
    assert it1.mean() < it0.mean() - 1.0, (it1.mean(), it0.mean())
    _, Tg = m.mlp_guess(te, tY)
    assert np.median(np.abs(Tg.cpu().numpy() - st.T)) < 30.0
    # the paper's FP64 Newton from the guess: fewer FP64 steps as well
    m64 = B.Mechanism(path, "newton=fp64")
    f = str(tmp_path / "guess.bin")
    m.mlp_save(f)
    m64.mlp_load(f)
    pa, na = m.mlp_get_params()
    pb, nb = m64.mlp_get_params()
    assert np.array_equal(pa, pb) and np.array_equal(na, nb)
    _, i64a = m64.temperature(te, tY, with_iters=True)
    T64, i64b = m64.temperature(te, tY, learned=True, with_iters=True)
    assert np.max(np.abs(T64.cpu().numpy() - oT) / oT) <= 1e-10
    assert i64b.double().mean().item() < i64a.double().mean().item() - 1.0


def test_learned_guess_requires_a_network(mech_files, dev):
    from paper_2503_24286_gb300 import binding as B
    m = B.Mechanism(mech_files[0][0])
    st = synth.config_states(0, n=16)
    orc = O.Oracle(mech_files[0][0])
    e = orc.internal_energy(st.T, st.Y)
    with pytest.raises(B.PyroError) as ei:
        m.temperature(_t(e, dev), _t(st.Y, dev), learned=True)
    assert ei.value.code == B.PYRO_ENOMLP
