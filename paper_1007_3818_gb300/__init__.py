"""GB300-native MUSCL-Hancock + Roe patch-group hydro step (paper Sec. 2).

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_1007_3818_gb300.native``.
"""
__all__ = ["native", "workloads"]
