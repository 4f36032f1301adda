"""Write the stored expected values of the GPU parity tests.

Calls only the CPU oracle (oracle/) on the seeded synthetic workloads of
paper_2602_14854_gb300.inputs and stores the final scalar flux and the stored
ranks per subdomain.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dd_dlra  # noqa: E402
from paper_2602_14854_gb300 import inputs  # noqa: E402


def main():
    wl = inputs.config_c1()
    t = time.time()
    o = dd_dlra.DDDLRA(wl)
    o.run()
    rho = o.scalar_flux()
    np.savez_compressed(os.path.join(HERE, "pointsource_128_rk4_t1.npz"), rho=rho,
                        ranks=np.array(o.ranks()), nsteps=wl.nsteps, dt=wl.dt)
    print(f"point source: {wl.nsteps} steps in {time.time() - t:.1f} s, ranks {o.ranks()}")


if __name__ == "__main__":
    main()
