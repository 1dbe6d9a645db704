"""Seeded synthetic image and mask generators (no inpainting arithmetic)."""
from .gen import *  # noqa: F401,F403
from .gen import __all__  # noqa: F401
