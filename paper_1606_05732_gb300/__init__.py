"""GB300-native CountGauss transform (Kapralov, Potluru, Woodruff, "How to Fake
Multiply by a Gaussian Matrix"): T.X = G.(S.X) with a CountSketch S and an
in-kernel Gaussian G, behind the C ABI of include/countgauss.h.

The CUDA library is loaded lazily on first use (``countgauss.CountGauss``); importing
the package does not touch the GPU.
"""
__all__ = ["countgauss", "synth", "build"]
