"""Write the converged-potential cache for the larger configurations.

Usage: python -m acp_workloads.make_cache [config ...]   (config 4: the 64 batched chains, SCF to
a density residual of 1e-4, several systems at a time)
Each cache file holds only V_eff (N_g doubles); loading it costs one dense eigensolve and is
checked against self-consistency before use, otherwise the SCF restarts from it.
"""
import sys
import time

from .ground_state import ground_state
from .systems import config


BATCH_SCF_TOL = 1e-4


def _batch_one(sysm):
    t = time.time()
    gs = ground_state(sysm, tol=BATCH_SCF_TOL)
    return f"{sysm.name}: N {sysm.n[0]} gap {gs.gap:.6f} residual {gs.scf_residual:.2e} " \
           f"iterations {gs.iterations} {time.time() - t:.1f}s"


def main(argv):
    for c in (argv or ["2"]):
        if int(c) == 4:
            import multiprocessing as mp
            from .systems import batch_config
            with mp.get_context("spawn").Pool(4) as pool:
                for line in pool.imap_unordered(_batch_one, sorted(batch_config(4), key=lambda s: -s.n[0])):
                    print(line, flush=True)
            continue
        sysm = config(int(c))
        t = time.time()
        gs = ground_state(sysm, verbose=True)
        print(f"{sysm.name}: gap {gs.gap:.6f} residual {gs.scf_residual:.2e} "
              f"iterations {gs.iterations} {time.time() - t:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:])
