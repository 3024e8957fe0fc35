"""FP64 CPU oracle (test infrastructure only; see ``qxd_oracle``)."""
from .qxd_oracle import *  # noqa: F401,F403
from .qxd_oracle import (CHARGE_C, CHARGE_C_INV, GAMMA, GAMMA5, PAULI, Dirac,  # noqa: F401
                         EvenOdd, GaugeField, Lattice, dense_matrix, gcr, sigma)
from .qxd_rhmc import (D_hat_dagger, cg, gamma5_mul, ln_abs_det_blocks,  # noqa: F401
                       ln_abs_det_Doo, normal_apply, pf_action_term, rational_apply,
                       shifted_solve)
from . import qxd_flow, qxd_rhmc  # noqa: F401
from . import qxd_dfl  # noqa: F401
