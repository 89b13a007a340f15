"""GB300-native kernel-compensated MFD Maxwell eigensolver for photonic crystals.

The numerical work runs in ``libpc.so`` (hand-written CUDA for sm_103a, C ABI declared in ``include/pc.h``). This
package is the thin Python binding over it: ``pc`` marshals arguments (numpy arrays for host buffers, torch CUDA
tensors for device buffers) and raises on any library error. There is no CPU fallback: importing the binding
without a built library raises.
"""
from .pc import (PCError, Solver, WarmStart, block_update, eigh_batched, eps_diamond, eps_gyroid, eps_spheres,
                 eps_spheres_lattice, gram, gram_pair, gram_pair_coupled, init_block, lattice_vectors, lib,
                 rayleigh_ritz, residual, stencil_coefficients)

__all__ = ["PCError", "Solver", "WarmStart", "block_update", "eigh_batched", "eps_diamond", "eps_gyroid",
           "eps_spheres", "eps_spheres_lattice", "gram", "gram_pair", "gram_pair_coupled", "init_block",
           "lattice_vectors", "lib", "rayleigh_ritz", "residual", "stencil_coefficients"]
