"""GB300-native CT volume ray caster (uniform cubic B-spline resampling, post-classification,
front-to-back compositing, early ray termination, brick empty-space leaping).

The rendering runs in hand-written CUDA kernels for sm_103a behind the C ABI of libvrc
(include/vrc.h); this package holds the kernels' sources (csrc/), the build step
(build.py), a ctypes binding (native.py), a thin context wrapper (renderer.py) and seeded
synthetic inputs (synth.py). Importing the package loads nothing; the library is loaded by
the first Renderer.
"""
__all__ = ["Renderer", "build", "native", "synth"]


def __getattr__(name):
    if name == "Renderer":
        from .renderer import Renderer
        return Renderer
    if name in ("build", "native", "synth"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
