"""GB300 FFT-convolution Poisson solver for free, wire, surface and periodic
boundary conditions (Dugan, Genovese, Goedecker: a customized zero-padding-aware
3D FFT). The compute path is the CUDA library ``lib/libpsolver.so`` behind the
C ABI in ``include/psolver.h``; ``psolver`` is its Python binding and
``autograd`` wraps it for torch.autograd."""

from .psolver import Plan, PsError, load_library, solve_batched  # noqa: F401
