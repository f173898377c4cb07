"""GB300-native CR-MC (charge-regulation Monte Carlo) hot path.

``paper_2109_07527_gb300.crmc`` is the Python binding of the C-ABI library
``libcrmc.so`` (hand-written sm_103a CUDA kernels); ``workloads`` builds the
seeded synthetic systems.  Importing the package does not load the CUDA
library; importing ``crmc`` does, and fails loudly if it is missing.
"""
__all__ = ["crmc", "workloads"]
