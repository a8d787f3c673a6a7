"""GB300-native speculative progressive isosurface raycasting (arXiv 2309.10212).

The renderer is the CUDA library libspr.so behind the C ABI in include/spr.h;
this package holds its sources (csrc/), its in-tree build (build.py) and a thin
Python binding with the same names as the C calls (api.py)."""
from .api import *  # noqa: F401,F403
from .api import Batch, Renderer, Server, Volume  # noqa: F401
from ._lib import SprError  # noqa: F401
