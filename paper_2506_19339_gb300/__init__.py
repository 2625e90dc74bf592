"""GB300-native split-CTMRG (arXiv:2506.19339): f and grad f of a 3D classical model from the
split corner-transfer renormalization group of the triple-layer PEPS-PEPO-PEPS network.

The compute lives in libsctm.so (CUDA, sm_103a) behind the C ABI of include/sctm.h; the Python
modules here only marshal arguments (``sctm``), build the library (``build``) and draw seeded
synthetic inputs (``inputs``).
"""
