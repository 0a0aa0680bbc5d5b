"""GB300 (sm_103a) multigrid ensemble Kalman filter (MGEnKF).

The compute path is the CUDA library ``libmgenkf.so`` (C ABI in
``include/mgenkf.h``); ``paper_2012_10091_gb300.mgenkf`` is its Python binding
and ``paper_2012_10091_gb300.workloads`` holds the seeded synthetic inputs.
Importing the binding raises if the library has not been built
(``python -m paper_2012_10091_gb300.build``).
"""

__all__ = ["build", "mgenkf", "workloads"]
