"""ctypes declarations of the boundary, geometry and structure entry points."""
from __future__ import annotations


def declare(L):
    pass
