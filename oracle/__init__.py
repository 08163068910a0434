"""CPU oracle of the traffic microsimulation (test infrastructure only).

Plain C (``oracle.c``) behind a thin ctypes wrapper.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import this package; the product
path (``paper_1807_01148_gb300``) never does.
"""
from .oracle import OracleSim, build, lib, oracle_idm, oracle_ballistic, oracle_link_cost, \
    oracle_sssp, oracle_mand_index, oracle_mand_tau, oracle_turn, oracle_signal_green, \
    oracle_reroute_selected, oracle_co_rate, oracle_fuel_rate  # noqa: F401
