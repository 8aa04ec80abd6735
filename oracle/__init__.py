"""FP64 CPU oracle for fKK-EC (test infrastructure only; see fkk_oracle)."""
from .fkk_oracle import *  # noqa: F401,F403
from .fkk_oracle import Basis, FitParams  # noqa: F401
