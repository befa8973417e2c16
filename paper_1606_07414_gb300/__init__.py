"""GB300-native 16-point multiplierless DCT-approximation codec (libtx16).

``paper_1606_07414_gb300.tx16`` is the ctypes binding of the C-ABI library
built from ``csrc/``; ``synth`` makes seeded synthetic inputs.  Importing the
package loads nothing: the CUDA library is loaded on first use of ``tx16``.
"""
