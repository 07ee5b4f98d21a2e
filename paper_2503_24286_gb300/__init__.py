"""GB300-native pointwise combustion thermochemistry (Pyrometheus formulation).

The compute path is the C-ABI library ``libpyro`` (mechanism-specialised CUDA
kernels for sm_103a); :mod:`.binding` marshals arguments to it.  Importing this
package loads nothing; :mod:`.synth` draws synthetic mechanisms and states.
"""
__all__ = ["synth"]
