"""GB300-native multi-hypothesis collision criticality (arXiv 2005.06773 hot path).

Importing the package does not load the CUDA library; ``paper_2005_06773_gb300.mhc`` does, and fails
loudly when it is missing.
"""
__all__ = ["scenarios"]
