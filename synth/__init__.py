"""Seeded synthetic inputs shared by the oracle-based tests and the device path.

Holds workload definitions (mesh hierarchy, field parameters, solver
settings) and seeded random test vectors. It contains none of the method's
arithmetic: no random-field, finite-element, solver or statistics code.
"""
from .workloads import WORKLOADS, workload, small_case, serving_request, serving_stream  # noqa: F401
from .vectors import random_node_vectors, random_element_field  # noqa: F401
