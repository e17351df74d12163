"""GB300-native docking hot path (Lamarckian GA over ligand poses).

``capi`` is the Python binding of the C-ABI library ``libdock.so`` (CUDA,
sm_103a); ``synth`` draws seeded synthetic inputs.  The binding loads the
CUDA library on first use and raises if it is missing: there is no CPU path.
"""
