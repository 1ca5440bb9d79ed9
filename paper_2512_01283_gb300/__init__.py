"""GB300-native polarized Monte-Carlo radiative transfer (Kratos-polrad method,
arXiv:2512.01283): C-ABI CUDA library ``libmcrt.so`` and its Python binding."""
from .mcrt import McrtError, Model, launch, lib, unit_eval  # noqa: F401
