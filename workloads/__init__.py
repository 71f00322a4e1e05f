"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path (no method arithmetic)."""
from .generators import *  # noqa: F401,F403
