"""Seeded synthetic inputs shared by the oracle tests and the CUDA parity tests.

Holds random draws and simple analytic test fields only: none of the method's
arithmetic (no deposit, FFT, force or growth computation) lives here.
"""
from .inputs import *  # noqa: F401,F403
