"""GB300-native hot path of the Blacklight ray tracer (White 2022, arXiv:2203.15963).

`native` is the ctypes binding of libblacklight.so (include/blacklight.h); `synth` builds the
seeded synthetic inputs; `images` allocates outputs and calls the binding for whole images.
"""
from . import synth  # noqa: F401
