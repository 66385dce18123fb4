"""FP64 CPU oracle of the incompressible DUGKS with force term (arXiv 1411.6121).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU-baseline /
reference legs import this package. The product path (``paper_1411_6121_gb300``) never
does, and shares no code with it.
"""
from .oracle import Oracle, OracleConfig, BC_PERIODIC, BC_NEQ_VELOCITY, BC_NEQ_PRESSURE  # noqa: F401
