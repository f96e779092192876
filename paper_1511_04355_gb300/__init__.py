"""GB300-native Laplace-domain elastodynamic BEM frequency solves (constant-element collocation,
matrix-free operator, batched GMRES with FP64 refinement, FSM, vector fitting, adaptive frequency
sampling).  The computation lives in the CUDA library built from csrc/ (see build.py); this package
only loads it and marshals arguments (binding.py)."""
from .binding import *  # noqa: F401,F403
from .binding import Context, BemError, load_library, declared_symbols  # noqa: F401
