"""B300-native coupled lattice Boltzmann electrohydrodynamics (LB-EHD) step.

The CUDA library (``liblbehd.so``) is loaded lazily by ``paper_2608_12868_b300.lbehd``;
importing the package itself touches no GPU code, so the input generators in
``workloads`` stay usable on machines without CUDA.
"""
__all__ = ["workloads", "lbehd"]
