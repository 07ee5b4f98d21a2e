import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def mech_dir(tmp_path_factory):
    return str(tmp_path_factory.mktemp("mechs"))


@pytest.fixture(scope="session")
def mech_files(mech_dir):
    """Synthetic workload mechanisms written once per session: {index: path} for the
    10-, 53-, 160-species mechanisms and the 53-species variant with SRI and PLOG (7)."""
    from paper_2503_24286_gb300 import synth
    out, objs = {}, {}
    for i in (0, 1, 4, 7):
        m = synth.config_mechanism(i)
        p = os.path.join(mech_dir, "mech%d.txt" % i)
        synth.write_mechanism(m, p)
        out[i], objs[i] = p, m
    return out, objs


@pytest.fixture(scope="session")
def mixed_reversibility_mech(mech_dir):
    """The 53-species SRI/PLOG variant with every third reaction made irreversible,
    so that reversible and irreversible reactions of each class sit side by side
    in the kernels' reaction order."""
    from paper_2503_24286_gb300 import synth
    m = synth.config_mechanism(7)
    for j, r in enumerate(m.reactions):
        if j % 3 == 1:
            r.reversible = False
    p = os.path.join(mech_dir, "mech7_mixed.txt")
    synth.write_mechanism(m, p)
    return p
