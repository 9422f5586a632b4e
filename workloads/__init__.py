"""Seeded synthetic inputs shared by the tests and the benchmark (no HyperIM arithmetic here)."""
from .hypergraphs import *  # noqa: F401,F403
