"""FP64 CPU oracle for the multipath Metropolis method (test infrastructure).

Only tests, the smoke check and the CPU-baseline leg of the bench import this
package.  The CUDA library never calls it and shares no code with it.

``run`` drives the C implementation in ``mp_oracle.c`` (paths run on host
threads); ``estimates`` turns its per-path records into the paper's ensemble
estimates with plain numpy.
"""
from .oracle import (  # noqa: F401
    CHAIN, ISING, SC, TWO_START, INIT_ANGLES, INIT_ORDERED, INIT_SPHERE, ORDER_CHECKER, ORDER_RANDOM,
    REC, NREC, System, build, energy, init, delta_e, philox, run, trial, lib_path,
)
from .estimates import estimates, distribution_coefficient  # noqa: F401
