"""Seeded input generators (meshes, flow conditions, initial fields) shared by the
CPU oracle tests and the CUDA path. Holds no arithmetic of the gas-kinetic method."""
