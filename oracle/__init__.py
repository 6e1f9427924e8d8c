"""FP64 CPU oracle (test infrastructure only; see ``vmat_oracle``)."""
from .vmat_oracle import *  # noqa: F401,F403
from .vmat_oracle import BBOptions, PlanResult  # noqa: F401
