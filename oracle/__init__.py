"""CPU FP64 oracle (test infrastructure only): see cncpd_oracle."""
from . import cncpd_oracle  # noqa: F401
