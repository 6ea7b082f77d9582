"""PPPM k-space particle-mesh path for GB300 (sm_103a).

Importing the package loads nothing native; ``paper_1702_04250_gb300.pppm``
loads the CUDA library and fails loudly if it has not been built.
"""
__all__ = ["workloads"]
