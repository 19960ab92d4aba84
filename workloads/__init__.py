"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the oracle.

This package holds none of the ICWF method's arithmetic.  It only tabulates model potentials
V(x, R) on the grids, diagonalises the electronic Hamiltonian for Born-Oppenheimer states (used
to build the initial state and as population projectors), and builds the initial wavefunction.
"""
from .models import (Workload, shin_metiu, cavity, shin_metiu_potential, cavity_potential,
                     bo_states, WORKLOADS)

__all__ = ["Workload", "shin_metiu", "cavity", "shin_metiu_potential", "cavity_potential",
           "bo_states", "WORKLOADS"]
