import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def oracle_pool(orc):
    """Worker processes for long oracle runs, so that they overlap the GPU
    work of the same tests.  Started with `spawn`: a worker forked from a
    process that has already initialised CUDA would hang."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = max(1, min(8, (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        yield ex


def oracle_config(orc, kw):
    """The oracle's Config for a run given as binding.make_config keywords."""
    pol = kw.get("policy", "steady")
    pol = orc.POLICY_NAMES[pol] if isinstance(pol, str) else pol
    return orc.Config(rows=kw.get("rows", 4), cols=kw.get("cols", 4), n=kw.get("n", 32),
                      tournament=kw.get("tournament", 2), policy=pol, bits=kw.get("bits", 1),
                      W=kw.get("W", 2), interval=kw.get("interval", 1),
                      p_ben=kw.get("p_ben", 0.0), p_del=kw.get("p_del", 0.0),
                      seed=kw.get("seed", 1), coarsen=kw.get("coarsen", 1))
