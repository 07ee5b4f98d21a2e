"""Point sharding: the path is pointwise (every state is independent, Sec. 4.4),
so evaluating two sub-ranges of the points in separate calls -- what each rank
does under data-parallel sharding -- must give results bit-identical to one call
over all points.  Checked for the forward path (internal-energy input: Newton +
omega), the JVP, the VJP and the dense Jacobian, with one thread per state and
with one warp per state.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_24286_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _split(a, cut):
    """The two point sub-ranges of an SoA array ([n] or [N][n]) as contiguous arrays."""
    return a[..., :cut].contiguous(), a[..., cut:].contiguous()


@pytest.mark.parametrize("opts", [None, "variant=warp"])
def test_two_shards_equal_one_call(mech_files, dev, opts):
    from paper_2503_24286_gb300 import binding as B
    from paper_2503_24286_gb300 import build as BLD
    BLD.build()
    path = mech_files[0][1]
    m = B.Mechanism(path, opts)
    orc = O.Oracle(path)
    n, cut = 1000, 377
    st = synth.config_states(1, n=n, offset_seed=91)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    rho, T, Y = t(orc.density(st.p, st.T, st.Y)), t(st.T), t(st.Y)
    e = m.internal_energy(T, Y)
    g = torch.Generator(device=dev).manual_seed(3)
    rnd = lambda *shape: torch.randn(shape, dtype=torch.float64, device=dev, generator=g)
    dr, dT, dY = rnd(n) * rho * 0.1, rnd(n), rnd(orc.N, n) * 1e-3
    u = rnd(orc.N, n)

    def calls(rho, T, Y, e, dr, dT, dY, u):
        w, Te = m.net_production_rates(rho, Y, e=e)
        out = [w, Te, m.jvp(rho, T, Y, dr, dT, dY), *m.vjp(rho, T, Y, u)]
        out.append(m.jacobian(rho, T, Y))
        return out

    full = calls(rho, T, Y, e, dr, dT, dY, u)
    parts = [_split(a, cut) for a in (rho, T, Y, e, dr, dT, dY, u)]
    a = calls(*[p[0] for p in parts])
    b = calls(*[p[1] for p in parts])
    torch.cuda.synchronize()
    for f, x, y in zip(full, a, b):
        assert torch.equal(f, torch.cat([x, y], dim=-1))
    assert m.nonconverged() == 0
