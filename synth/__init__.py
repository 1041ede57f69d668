"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package holds input distributions only: molecular-shaped one- and
two-electron integrals, random statevectors, random ansatz draws and the
serving request stream.  It contains none of the method's arithmetic (no
qubit mapping, no Pauli algebra, no state evolution), so that importing it
from both sides of a parity test does not couple them.
"""

from .integrals import (  # noqa: F401
    Integrals,
    molecular_integrals,
    CONFIGS,
    config_integrals,
)
from .draws import (  # noqa: F401
    random_state,
    draw_ansatz,
    serving_requests,
    ServingRequest,
)
