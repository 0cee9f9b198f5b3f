"""Plain FP64 CPU oracle of the AMR ideal-MHD level advance.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg; never by the product package.
"""
from .oracle import OracleSim, build_map, hlld, mhd_flux, minmod, fast_speed, gs_edge, MAPS  # noqa: F401
