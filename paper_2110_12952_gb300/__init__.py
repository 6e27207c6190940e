"""GB300 library for cellular automata on NBB fractals in compact storage.

Implements the data-parallel hot path of Quezada & Navarro, "Accelerating
Compact Fractals with Tensor Core GPUs" (2021): the thread maps lambda
(compact -> embedded) and nu (embedded -> compact, Sec. 3.1), and the
stencil step that combines them (Sec. 3), next to the bounding-box baseline
(Sec. 4).  The compute runs in hand-written CUDA kernels for sm_103a behind
the C ABI of ``include/fractal.h``; ``Fractal`` is its Python binding.

Importing the package does not load the CUDA library; the first ``Fractal``
does, and raises if ``libfractal.so`` has not been built.
"""

__all__ = ["Fractal", "Batch", "Server", "FractalError", "build", "workloads"]


def __getattr__(name):
    if name == "Fractal":
        from .fractal import Fractal
        return Fractal
    if name == "Batch":
        from .fractal import Batch
        return Batch
    if name == "Server":
        from .fractal import Server
        return Server
    if name == "FractalError":
        from .capi import FractalError
        return FractalError
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
