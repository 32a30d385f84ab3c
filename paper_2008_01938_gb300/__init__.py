"""Exact GB300 (sm_103a) solvers for the dynamic programs of Matsumae &
Miyazaki, "Solving Dynamic Programming Problem by Pipeline Implementation on
GPU": the matrix-chain multiplication table (Section IV-A, Eq. (2)) and the
simplified DP problem (Definition 1, Eq. (1)).

The computation runs in the CUDA kernels of ``libdpgpu.so`` behind the C ABI
of ``include/dpgpu.h``; the functions here only marshal PyTorch tensors
(device memory, streams) into those calls.  Importing this package does not
load the library; the first solver call does, and fails loudly if the library
has not been built.
"""
from .api import (  # noqa: F401
    McmPlan,
    SdpPlan,
    Server,
    interval_dp_solve,
    mcm_solve,
    mcm_solve_host,
    mcm_traceback,
    sdp_solve,
    sdp_solve_host,
    sync_status,
)
