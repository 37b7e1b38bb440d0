"""FP64 CPU oracle for the pSRM EM iteration (``psrm``; ``init``: Algorithm
1's random orthogonal W^0 drawn from a seed, as the library draws it) and the HTFA
local-step evaluations (``htfa``: the factor matrix of Eq. 14, the
residual of the local objective and the z-score).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call,
link or run anything in this package; only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline / reference arm of ``bench.py`` use
it.  It shares no code with the CUDA path.
"""
from .psrm import (  # noqa: F401
    center,
    estep,
    estep_dense,
    loglik,
    loglik_dense,
    sigma_update,
    polar_factor,
    mstep,
    fit,
    transform,
    map_subjects,
    ppca_fixed_point,
    State,
)
from .htfa import rbf_factors, residual as htfa_residual, residual_batch as htfa_residual_batch, zscore  # noqa: F401,E402
from .init import haar_w0, philox4x64_10, standard_normals  # noqa: F401,E402
