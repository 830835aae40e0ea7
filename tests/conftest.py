import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# tests/test_oracle_mutants.py runs the oracle's pins against a copy of the
# oracle with one planted mistake: that copy's parent directory goes first
if os.environ.get("FSB_MUTANT_ORACLE_PARENT"):
    sys.path.insert(0, os.environ["FSB_MUTANT_ORACLE_PARENT"])


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfsb.so")
    config.addinivalue_line(
        "markers", "slow: long-running case")
