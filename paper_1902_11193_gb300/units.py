"""Unit conversion for reporting (Sec. 4.3): a permeability in lattice units
times the squared voxel size is an area; one Darcy is 9.869233e-13 m^2 (the
paper's factor 0.9869 is one Darcy in square micrometres)."""

DARCY_M2 = 9.869233e-13


def darcy_from_lattice(k_lb: float, dx_m: float) -> float:
    """k in Darcy from k in lattice units at voxel size dx (metres)."""
    return k_lb * dx_m * dx_m / DARCY_M2


def lattice_from_darcy(k_D: float, dx_m: float) -> float:
    return k_D * DARCY_M2 / (dx_m * dx_m)
