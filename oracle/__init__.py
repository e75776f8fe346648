"""FP64 CPU oracle (test infrastructure only; see galario_oracle)."""
from .galario_oracle import *  # noqa: F401,F403
from .galario_oracle import __all__  # noqa: F401
