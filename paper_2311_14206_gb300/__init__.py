"""GB300-native GMRES-SDR: C-ABI library libsdr.so plus a thin ctypes binding.

GMRES with randomized sketching and deflated restarting (Burke, Guettel,
Soodhalter): truncated Arnoldi, a hash-defined sparse-sign embedding, a
sketched least-squares solve and sketched harmonic-Ritz recycling, each step
a hand-written sm_103a kernel.
"""
from .sdr import (  # noqa: F401
    SDR_PREC_F32_REFINED,
    SDR_PREC_F64,
    CSRDevice,
    Solver,
    SdrError,
    load_library,
    make_params,
    sdr_create,
    sdr_destroy,
    sdr_get_history,
    sdr_get_givens,
    sdr_set_sketch_draws,
    sdr_profile,
    sdr_profile_get,
    sdr_trace,
    sdr_trace_get,
    sdr_recycle,
    sdr_recycle_dim,
    sdr_recycle_export,
    sdr_recycle_import,
    sdr_sketch,
    sdr_sketch_noalloc,
    sdr_recycle_batch,
    sdr_solve,
    sdr_solve_batch,
)
from .adjoint import AdjointPair, SDRSolve  # noqa: F401,E402
