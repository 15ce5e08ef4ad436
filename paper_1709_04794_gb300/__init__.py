"""GB300-native fast binary semi-supervised discriminant analysis (FSDA).

The solver lives in the C-ABI library ``libsda.so`` (CUDA kernels for
sm_103a); :mod:`.sda` is its thin Python binding and :mod:`.synth` the
seeded input generator.  Importing the package loads nothing native; the
binding raises as soon as it is used without the built library.
"""
__all__ = ["sda", "synth"]
