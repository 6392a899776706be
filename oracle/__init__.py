"""FP64 CPU oracle of the quadric rasterizer: test infrastructure only (see qgs_oracle)."""
from .qgs_oracle import *  # noqa: F401,F403
