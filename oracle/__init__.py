"""FP64 CPU oracle (test infrastructure; see ``oracle.tucker_fp64``)."""
from .tucker_fp64 import *  # noqa: F401,F403
