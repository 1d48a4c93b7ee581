"""CPU oracle package — test infrastructure only (see ``crp_oracle``)."""
from .crp_oracle import *  # noqa: F401,F403
from . import crp_oracle  # noqa: F401
