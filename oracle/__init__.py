"""CPU oracle (test infrastructure only): see ``oracle.dsm_oracle``."""
from .dsm_oracle import *  # noqa: F401,F403
