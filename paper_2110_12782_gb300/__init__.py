"""GB300-native SketchNE hot path.

Submodules (imported explicitly, so that the seeded inputs can be used without
the CUDA library):

* ``paper_2110_12782_gb300.sketchne``: ctypes binding of ``libsketchne.so``.
* ``paper_2110_12782_gb300.synth``: seeded synthetic graphs.
* ``paper_2110_12782_gb300.build``: compiles the library for sm_103a.
"""
