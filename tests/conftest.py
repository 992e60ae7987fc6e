import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

# oracle jobs of the full-size parity tests (tests/oracle_jobs.py), started in worker
# processes as soon as the tests that use them are collected, so that their minutes of
# CPU work overlap the rest of the GPU run
_JOB_POOL = None
_JOB_FUTURES = {}
_JOB_USERS = {"test_gpu_z_configs.py": ("c2_run", "c3_run", "c5_phi_adj", "c5_iteration")}


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests need a device; they are selected with -m gpu and fail loudly if the
    # library or the device is missing, so nothing here skips them silently.
    pass


def pytest_collection_finish(session):
    global _JOB_POOL
    if session.config.option.collectonly:
        return
    wanted = []
    for item in session.items:
        base = os.path.basename(str(item.fspath))
        for name in _JOB_USERS.get(base, ()):
            if name not in wanted:
                wanted.append(name)
    if not wanted:
        return
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle_jobs
    # spawn: the workers start clean (no CUDA context is inherited) and import only
    # the oracle and the input generators
    _JOB_POOL = cf.ProcessPoolExecutor(max_workers=len(wanted), mp_context=mp.get_context("spawn"))
    for name in wanted:
        _JOB_FUTURES[name] = _JOB_POOL.submit(oracle_jobs.run, name)


def pytest_sessionfinish(session, exitstatus):
    if _JOB_POOL is not None:
        _JOB_POOL.shutdown(wait=False, cancel_futures=True)


@pytest.fixture(scope="session")
def oracle_job():
    """oracle_job(name) -> the result of oracle_jobs.run(name), computed in the session's
    worker pool when it was started, otherwise here."""
    import oracle_jobs
    cache = {}

    def get(name):
        if name not in cache:
            fut = _JOB_FUTURES.get(name)
            cache[name] = fut.result() if fut is not None else oracle_jobs.run(name)
        return cache[name]
    return get
