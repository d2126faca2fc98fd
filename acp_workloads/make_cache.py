"""Write the converged-potential cache for the larger configurations.

Usage: python -m acp_workloads.make_cache [config ...]
Each cache file holds only V_eff (N_g doubles); loading it costs one dense eigensolve and is
checked against self-consistency before use, otherwise the SCF restarts from it.
"""
import sys
import time

from .ground_state import ground_state
from .systems import config


def main(argv):
    for c in (argv or ["2"]):
        sysm = config(int(c))
        t = time.time()
        gs = ground_state(sysm, verbose=True)
        print(f"{sysm.name}: gap {gs.gap:.6f} residual {gs.scf_residual:.2e} "
              f"iterations {gs.iterations} {time.time() - t:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:])
