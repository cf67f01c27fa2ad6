"""GB300-native GW self-energy evaluation (density-fitted scGW hot path).

Importing the package loads nothing compiled. The CUDA library is loaded by
``paper_2406_18479_gb300.gw`` on first use and raises if it is missing.
"""
__version__ = "0.1.0"
