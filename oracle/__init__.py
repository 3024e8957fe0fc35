"""FP64 CPU oracle (test infrastructure only; see ``qxd_oracle``)."""
from .qxd_oracle import *  # noqa: F401,F403
from .qxd_oracle import (CHARGE_C, CHARGE_C_INV, GAMMA, GAMMA5, PAULI, Dirac,  # noqa: F401
                         EvenOdd, GaugeField, Lattice, dense_matrix, gcr, sigma)
