"""GB300-native quantization-aware interpolation (``qai``).

``paper_2602_20097_gb300.qai`` is the Python binding of the C-ABI library
``libqai.so`` (hand-written sm_103a CUDA kernels); ``synth`` makes seeded
synthetic inputs.
"""
