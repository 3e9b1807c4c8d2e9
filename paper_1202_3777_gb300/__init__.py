"""GB300-native junction-tree belief propagation.

Each Hugin message (marginalise a clique onto its separator, form the
new/old separator ratio, scatter-multiply it into the neighbour; Eq. 1-3)
runs in hand-written CUDA kernels for sm_103a behind the C ABI declared in
``include/jt.h``.  :mod:`paper_1202_3777_gb300.jt` is the thin ctypes binding
(same names as the C entry points); :mod:`paper_1202_3777_gb300.synth` builds
seeded synthetic trees and evidence.
"""
