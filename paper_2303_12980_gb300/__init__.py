"""GB300-native GMP (Gaussian Multipole) featurization behind a C ABI.

`binding` loads libgmp.so (CUDA, sm_103a) lazily; `synth` holds the seeded
synthetic workloads; `build` compiles the library in-tree.
"""
__all__ = ["binding", "synth", "build"]


def __getattr__(name):
    if name in ("GMPFeaturizer", "gmp_features", "GMPError", "load_library"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
