"""GB300-native AICA pair-force path (Arbitrary Interacting Cells Algorithm).

The compute path lives in the CUDA library ``libaica.so`` built from
``csrc/``; :mod:`paper_cs_0702131_gb300.aica` is its thin ctypes binding and
loads it on first use.  :mod:`paper_cs_0702131_gb300.synth` builds seeded
synthetic inputs and loads nothing.
"""
