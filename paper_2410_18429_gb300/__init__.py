"""GB300-native hot path of source-free adaptive Wavefield Reconstruction Inversion.

The CUDA kernels live in ``csrc/`` and are built into ``libwri.so`` (C ABI declared in
``include/wri.h``); :mod:`.wri` is the ctypes binding (importing it raises if the
library is missing), :mod:`.problem` moves seeded inputs onto the device,
:mod:`.objective` wraps the reduced objective as a ``torch.autograd.Function``,
:mod:`.awri` runs the adaptive outer loop (Algorithm 2), :mod:`.grids` maps one model onto the
frequency groups' own grids, and :mod:`.parallel_sum` holds the gradient sum over ranks of a
sharded evaluation.
"""
_API = ("C64", "C128", "GroupSpec", "apply_A", "autotune", "gradient", "gradient_noalloc", "make_opts", "solve",
        "source_estimate", "workspace_size")


def __getattr__(name):
    if name in _API:
        from . import wri
        return getattr(wri, name)
    raise AttributeError(name)
