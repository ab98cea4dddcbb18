"""lsyn: GB300-native bottom-up semantic enumeration of LTLf formulae.

The compute path is a C-ABI CUDA library (``csrc/``, declared in
``include/lsyn.h``); ``paper_2504_18943_gb300.lsyn`` is its thin Python
binding. ``workloads`` holds the seeded synthetic input generators.
"""
