"""GB300-native density-matrix engine for noisy quantum-device emulation (libvqd + binding)."""
from . import vqd  # noqa: F401
from .vqd import *  # noqa: F401,F403
