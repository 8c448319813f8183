"""FP64 CPU oracle (test infrastructure only; see ``spmttkrp_oracle``)."""
from .spmttkrp_oracle import *  # noqa: F401,F403
