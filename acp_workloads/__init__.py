"""Seeded input generators shared by the CPU oracle and the CUDA path (no method arithmetic)."""
from .systems import System, config, paper_chain, small_chain, mixed_chain, chain_1d, srft_sketch  # noqa: F401
from .ground_state import GroundState, ground_state, scf  # noqa: F401
