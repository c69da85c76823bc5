"""Seeded synthetic inputs (graphs and caller colourings) shared by the
oracle's tests and the CUDA path's tests and benchmark."""
from .graphs import *  # noqa: F401,F403
from .graphs import CSRGraph, from_edges  # noqa: F401
