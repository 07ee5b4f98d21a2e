"""Small hand-built mechanisms for special-case tests (closed forms by hand)."""
import os

from paper_2503_24286_gb300 import synth


def const_cp_species(name, comp, a1, a6, a7):
    """cp/R = a1 (constant): h/RT = a1 + a6/T, s/R = a1 ln T + a7 in both ranges."""
    c = [a1, 0.0, 0.0, 0.0, 0.0, a6, a7]
    return synth.Species(name, comp, list(c), list(c))


def write(mech, directory, fname):
    p = os.path.join(directory, fname)
    synth.write_mechanism(mech, p)
    return p


def abcd_mechanism(kind="arrhenius", A=1e10, b=0.5, theta=5000.0, eff=None, low=None, troe=None,
                   a6=(0.0, 0.0, 0.0, 0.0)):
    """A + B <=> C + D over one element-free 'X' bookkeeping: A=X, B=X2 -> C=X2... balanced:
    species X (1 atom), Y2 (2 atoms), XY (1+1) ... here: H + O2 <=> OH + O."""
    els = [("H", synth.ATOMIC_WEIGHTS["H"]), ("O", synth.ATOMIC_WEIGHTS["O"])]
    sp = [const_cp_species("H", {"H": 1}, 2.5, a6[0], 10.0),
          const_cp_species("O2", {"O": 2}, 3.5, a6[1], 12.0),
          const_cp_species("OH", {"H": 1, "O": 1}, 3.5, a6[2], 11.0),
          const_cp_species("O", {"O": 1}, 2.5, a6[3], 9.0)]
    r = synth.Reaction(kind, [(0, 1), (1, 1)], [(2, 1), (3, 1)], A, b, theta,
                       efficiencies=dict(eff or {}), low=low, troe=troe)
    return synth.Mechanism("abcd", els, sp, [r])
