"""Seeded input generators shared by the CPU oracle and the CUDA path (no method arithmetic)."""
from .systems import (System, batch_config, chain_1d, config, lattice_2d, mixed_chain, paper_chain,  # noqa: F401
                      small_chain, small_lattice, smooth_5, srft_sketch, training_lattices)
from .ground_state import GroundState, ground_state, scf  # noqa: F401
from . import learned  # noqa: F401
