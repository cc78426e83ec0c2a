import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: oracle runs that take more than a few seconds")


@pytest.fixture(scope="session")
def c1():
    """4x4 TFIM h=3.0, m=8, 4 disentanglers, seed 0 (the small FP64 workload)."""
    from oracle.lattice import square_lattice, tfim_terms
    from oracle.tree import Tree
    from oracle.disentangle import place_disentanglers

    lat = square_lattice(4)
    terms = tfim_terms(lat, 3.0)
    tree = Tree(16, 8)
    des = place_disentanglers(tree, terms, 4)
    return lat, terms, tree, des
