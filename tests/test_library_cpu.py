"""Host-side checks of libpyro that need no GPU: the library loads, exports every
symbol declared in include/pyro.h, parses and validates mechanisms, emits and
compiles (NVRTC, sm_103a) the specialised kernels, and rejects bad input."""
import ctypes
import os
import re

import pytest

from paper_2503_24286_gb300 import binding as B
from paper_2503_24286_gb300 import build as BLD
from paper_2503_24286_gb300 import synth
from tests import handmech

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built(tmp_path_factory):
    os.environ.setdefault("PYRO_CACHE_DIR", str(tmp_path_factory.mktemp("jit")))
    BLD.build()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pyro_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.LIB_PATH)
    declared = _declared()
    assert {"pyro_mech_load", "pyro_temperature", "pyro_net_production_rates"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(B.EXPORTS) == declared
    assert B.lib().pyro_version() >= 100


def test_compile_only_handle_and_static_counts(mech_files):
    paths, objs = mech_files
    m = B.Mechanism(paths[0], "device=0")
    assert (m.n_species, m.n_reactions) == (10, 21)
    W = [sum(c * synth.ATOMIC_WEIGHTS[e] for e, c in s.composition.items()) for s in objs[0].species]
    assert m.W == pytest.approx(W, rel=1e-15)
    assert m.stat("omega_fp64_flops_per_point") > 0
    assert m.stat("cubin_bytes") > 1000
    src = m.source()
    assert "pyro_omega" in src and "pyro_tsolve" in src
    # a compile-only handle cannot launch
    import numpy as np
    with pytest.raises(B.PyroError) as ei:
        m.internal_energy(np.ones(4), np.ones((10, 4)) / 10)
    assert ei.value.code == B.PYRO_EINVAL


def test_derivative_kernels_compile_without_gpu(mech_files):
    m = B.Mechanism(mech_files[0][0], "device=0")
    m.prepare("jvp,vjp,jacobian")
    for g in ("jvp", "vjp", "jac"):
        assert m.stat(g + "_cubin_bytes") > 1000
    assert m.stat("jacobian_scratch_doubles_per_point") > 0
    with pytest.raises(B.PyroError):
        m.prepare("hessian")


def test_adiabatic_jacobian_and_crank_nicolson_kernels_compile_without_gpu(mech_files):
    m = B.Mechanism(mech_files[0][0], "device=0")
    m.prepare("jacobian_adiabatic,cn")
    assert m.stat("jad_cubin_bytes") > 1000 and m.stat("cn_cubin_bytes") > 1000
    L = B.lib()
    D = ctypes.POINTER(ctypes.c_double)
    x = (ctypes.c_double * 40)()
    px = ctypes.cast(x, D)
    # argument checks come before any device work: bad dt / tol / max_newton, null arrays
    assert L.pyro_cn_step(m.handle, 4, -1.0, px, px, px, 1e-12, 20, px, px, None, None) == B.PYRO_EINVAL
    assert L.pyro_cn_step(m.handle, 4, 1e-9, px, px, px, 0.0, 20, px, px, None, None) == B.PYRO_EINVAL
    assert L.pyro_cn_step(m.handle, 4, 1e-9, px, px, px, 1e-12, 0, px, px, None, None) == B.PYRO_EINVAL
    assert L.pyro_cn_step(m.handle, 4, 1e-9, None, px, px, 1e-12, 20, px, px, None, None) == B.PYRO_EINVAL
    assert L.pyro_cn_step(m.handle, 0, 1e-9, None, None, None, 1e-12, 20, None, None, None, None) == B.PYRO_OK
    assert L.pyro_jacobian_adiabatic(m.handle, 4, None, px, px, px, None) == B.PYRO_EINVAL


def test_table_row_jacobian_kernels_compile_without_gpu(mech_files):
    """Jacobian rows from emitted tables (the assembly large mechanisms use), with the
    per-state species arrays in the global scratch (store=global): the Jacobian,
    dS/dY and Crank-Nicolson units compile; the scratch holds the slots plus the two
    species arrays; the solve takes four states per block at 10 species."""
    m = B.Mechanism(mech_files[0][0], "device=0;jac_rows=table;store=global")
    m.prepare("jacobian,jacobian_adiabatic,cn")
    assert m.stat("jacobian_rows_from_tables") == 1 and m.stat("deriv_store_global") == 1
    assert m.stat("jac_cubin_bytes") > 1000 and m.stat("jad_cubin_bytes") > 1000 and m.stat("cn_cubin_bytes") > 1000
    inline = B.Mechanism(mech_files[0][0], "device=0")
    assert inline.stat("jacobian_rows_from_tables") == 0
    assert m.stat("jacobian_scratch_doubles_per_point") == inline.stat("jacobian_scratch_doubles_per_point") + 2 * 10
    assert m.stat("cn_solve_warps") == 4


def test_transport_kernels_compile_without_gpu(mech_files, tmp_path):
    m = B.Mechanism(mech_files[0][0], "device=0")
    assert m.stat("has_transport") == 1
    m.prepare("transport")
    assert m.stat("tr_cubin_bytes") > 1000 and m.stat("transport_fp64_ops_per_point") > 0
    L = B.lib()
    D = ctypes.POINTER(ctypes.c_double)
    x = ctypes.cast((ctypes.c_double * 40)(), D)
    assert L.pyro_transport(m.handle, 4, x, x, None, None, None, None) == B.PYRO_EINVAL   # no output
    assert L.pyro_transport(m.handle, 4, None, x, x, None, None, None) == B.PYRO_EINVAL
    # a mechanism file without a transport section: no transport kernels, PYRO_EMECH
    mb = B.Mechanism(handmech.write(handmech.abcd_mechanism(), str(tmp_path), "abcd.txt"), "device=0")
    assert mb.stat("has_transport") == 0
    assert L.pyro_transport(mb.handle, 4, x, x, x, None, None, None) == B.PYRO_EMECH
    with pytest.raises(B.PyroError):
        mb.prepare("transport")


def test_pressure_dependent_forms_parse_validate_and_compile(mech_files, tmp_path):
    m = B.Mechanism(mech_files[0][7], "device=0")
    assert m.stat("omega_fp64_flops_per_point") > 0
    src = m.source()
    assert "(plog)" in src and "lnp" in src
    # the warp-per-state kernel is emitted for SRI and PLOG reactions too, and compiles
    mw = B.Mechanism(mech_files[0][7], "device=0;variant=warp;cache=0")
    mw.prepare("warp")
    assert mw.stat("wfwd_cubin_bytes") > 0 and mw.stat("warp_chunks") >= 325 / 32
    # and the block-per-state Jacobians (clusters of 4 states), with the reaction
    # chunks spread evenly enough over the 8 warps
    mw.prepare("jacobian,jacobian_adiabatic")
    assert mw.stat("jacobian_cta") == 1 and mw.stat("jacobian_adiabatic_cta") == 1
    assert mw.stat("wjac_cubin_bytes") > 0 and mw.stat("wjad_cubin_bytes") > 0
    assert mw.stat("wjac_nonzeros") <= 53 * 53 and mw.stat("wjac_terms") >= mw.stat("wjac_nonzeros")
    assert mw.stat("wjac_reaction_phase_imbalance") < 2.5
    # the warp tables pack three factors a side: a fourth-order reaction is refused
    # by variant=warp (and accepted by the thread-per-state kernels)
    mech = handmech.abcd_mechanism()
    mech.reactions[0].reactants = [(0, 2), (1, 2)]
    mech.reactions[0].products = [(2, 2), (3, 2)]
    p4 = handmech.write(mech, str(tmp_path), "order4.txt")
    assert B.Mechanism(p4, "device=0").stat("omega_fp64_flops_per_point") > 0
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(p4, "device=0;variant=warp")
    assert ei.value.code == B.PYRO_EINVAL and "three factors" in str(ei.value)
    # one NASA range choice per state: species with another T_mid are refused too
    mech = handmech.abcd_mechanism()
    mech.species[1].t_mid = 1500.0
    pt = handmech.write(mech, str(tmp_path), "tmid.txt")
    assert B.Mechanism(pt, "device=0").stat("jacobian_supported") == 0
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(pt, "device=0;variant=warp")
    assert ei.value.code == B.PYRO_EINVAL and "T_mid" in str(ei.value)
    mech = handmech.abcd_mechanism(kind="falloff", low=(1e16, -1.0, 1000.0))
    mech.reactions[0].sri = (0.5, 100.0, -3.0)                # c must be positive
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(handmech.write(mech, str(tmp_path), "badsri.txt"), "device=0")
    assert ei.value.code == B.PYRO_EMECH
    mech = handmech.abcd_mechanism()
    mech.reactions[0].kind = "plog"
    mech.reactions[0].plog = [(1e5, 1e10, 0.0, 100.0), (1e4, 1e10, 0.0, 100.0)]   # decreasing pressures
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(handmech.write(mech, str(tmp_path), "badplog.txt"), "device=0")
    assert ei.value.code == B.PYRO_EMECH


def test_unbalanced_mechanism_is_rejected(tmp_path):
    mech = handmech.abcd_mechanism()
    mech.reactions[0].products = [(2, 1), (3, 2)]      # H + O2 -> OH + 2 O : O not balanced
    p = handmech.write(mech, str(tmp_path), "bad.txt")
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(p, "device=0")
    assert ei.value.code == B.PYRO_EMECH
    assert "balanced" in str(ei.value)


def test_missing_file_and_bad_options(tmp_path, mech_files):
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(str(tmp_path / "nope.txt"), "device=0")
    assert ei.value.code == B.PYRO_EMECH
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(mech_files[0][0], "device=0;block=33")
    assert ei.value.code == B.PYRO_EINVAL
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(mech_files[0][0], "device=0;frobnicate=1")
    assert ei.value.code == B.PYRO_EINVAL
    for bad in ("cn_newton=quasi", "cn_refresh=0", "cn_refresh=5000", "jac_rows=sparse"):
        with pytest.raises(B.PyroError) as ei:
            B.Mechanism(mech_files[0][0], "device=0;" + bad)
        assert ei.value.code == B.PYRO_EINVAL
    B.Mechanism(mech_files[0][0], "device=0;cn_newton=chord;cn_refresh=8").close()


def test_cp_margin_validation(tmp_path):
    mech = handmech.abcd_mechanism()
    mech.species[0].nasa_low[0] = 0.5          # cp/R = 0.5 < 1: c_v < 0
    mech.species[0].nasa_high[0] = 0.5
    p = handmech.write(mech, str(tmp_path), "cp.txt")
    with pytest.raises(B.PyroError) as ei:
        B.Mechanism(p, "device=0")
    assert ei.value.code == B.PYRO_EMECH


def test_null_and_negative_arguments_rejected(mech_files):
    L = B.lib()
    h = ctypes.c_void_p()
    assert L.pyro_mech_load(None, None, ctypes.byref(h)) == B.PYRO_EINVAL
    m = B.Mechanism(mech_files[0][0], "device=0")
    assert L.pyro_density(m.handle, -1, None, None, None, None, None) == B.PYRO_EINVAL
    assert L.pyro_temperature(m.handle, 4, None, None, None, 0, None, None, None) == B.PYRO_EINVAL
    # n == 0 is a no-op even without pointers
    assert L.pyro_net_production_rates(m.handle, 0, None, None, 0, None, None, None, None) == B.PYRO_OK


def test_concurrent_loads_emit_the_same_sources(mech_files, tmp_path):
    """Separate handles are independent: mechanisms loaded from several host
    threads at once get exactly the sources a single load emits (the emitters'
    per-emission settings -- e.g. the accumulators-in-memory mode of mechanisms
    above 64 species -- must not leak between concurrent loads)."""
    import threading
    from paper_2503_24286_gb300 import synth
    paths, _ = mech_files
    big = synth.generate_mechanism("big70", ["C", "H", "O", "N"], 70, 60, 6, 4, 0, [], seed=11)
    paths = {1: paths[1], 4: str(tmp_path / "big70.txt")}
    synth.write_mechanism(big, paths[4])
    ref = {i: B.Mechanism(paths[i], "device=0").source() for i in (1, 4)}
    assert "Wp[" in ref[4] and "Wp[" not in ref[1]      # accumulators in memory only above 64 species
    got, errs = [], []

    def load(i):
        try:
            got.append((i, B.Mechanism(paths[i], "device=0").source()))
        except Exception as e:          # pragma: no cover - reported below
            errs.append(repr(e))
    th = [threading.Thread(target=load, args=(i,)) for i in (1, 4, 1, 4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs
    assert len(got) == 4 and all(src == ref[i] for i, src in got)
