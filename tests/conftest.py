"""Shared pytest configuration.

``-m gpu`` selects the parity tests that need a GB300 (CUDA); everything else
runs on the CPU.  The repository root is put on ``sys.path`` so that the
tests import ``oracle``, ``synthetic`` and the product package in-tree.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

R_EARTH = 6371220.0


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    return oracle


_MESHES = {}


@pytest.fixture(scope="session")
def omesh():
    """Factory of cached oracle meshes keyed by N."""
    from oracle.oracle import Mesh

    def get(N):
        if N not in _MESHES:
            _MESHES[N] = Mesh(N, R_EARTH)
        return _MESHES[N]

    return get


@pytest.fixture(scope="session")
def product():
    """The product package with its library built in-tree (nvcc, no GPU needed)."""
    from paper_1908_07038_gb300 import build as pbuild
    pbuild.build()
    from paper_1908_07038_gb300 import atlas, capi
    return atlas, capi


_FVMS = {}


@pytest.fixture(scope="session")
def pfvm(product):
    """Factory of cached product Fvm objects keyed by N."""
    atlas, _ = product

    def get(N):
        if N not in _FVMS:
            _FVMS[N] = atlas.build_fvm(N, R_EARTH)
        return _FVMS[N]

    return get
