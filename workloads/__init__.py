"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

Geometry/tag builders (``meshes``) and counter-based sample-parameter draws
(``params``).  Nothing here evaluates the method (no assembly, no solves):
these modules only produce the input arrays.  ``configs`` names the standard
workloads with their sizes.
"""
from . import meshes, params, configs  # noqa: F401
