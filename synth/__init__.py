"""Seeded synthetic inputs for the NOLSM density step.

This package builds the sparse one-particle Hamiltonian H0 and overlap S of
model systems (water boxes, a protein-like globule), the column blocks and
the geometric neighbourhood lists.  It holds none of the method's arithmetic
(no index-set rule, no matrix function, no trace): both the CUDA path and the
CPU oracle take its output as plain arrays.
"""
from .system import System, CONFIGS, make_config, water_box, water_clusters, isolated_waters, dimer_system, dense_blocks, protein_globule, atom_blocks, displaced  # noqa: F401
