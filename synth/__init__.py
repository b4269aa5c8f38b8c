"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests
and the benchmark.  This package holds none of the method's arithmetic: it
only draws seeded random numbers and simple spatial profiles."""
from .inputs import *  # noqa: F401,F403
