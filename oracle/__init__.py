"""Plain CPU oracle of the divide-and-merge graph-index build (test infrastructure only)."""
from .oracle import *  # noqa: F401,F403
