"""GB300-native Projected Adam estimator of the L2 condition number.

Importing the package is cheap: the CUDA binding is loaded on first use of
``paper_2409_11515_gb300.pa``.
"""
__all__ = ["synth", "pa"]
