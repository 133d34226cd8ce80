"""The oracle's pins catch plausible mistakes: each mistake of tests/oracle_mutants.py is planted in the
oracle, on the CPU, in a child pytest process of its own, and at least one of its pin tests must fail
there (pytest exit status 1: a test failed, or its fixture raised), while the same pins pass in the unmodified oracle (they run
in the main session).  The children run side by side, one BLAS thread each."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from tests import oracle_mutants

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(name):
    pins = oracle_mutants.MUTANTS[name][2]
    env = dict(os.environ, ORACLE_MUTANT=name, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "tests.oracle_mutants", "-p", "no:cacheprovider",
           "-m", "not gpu", *pins]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-3000:] + p.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes():
    names = list(oracle_mutants.MUTANTS)
    workers = max(1, min(len(names), os.cpu_count() or 1, 16))
    with ThreadPoolExecutor(workers) as ex:
        return dict(zip(names, ex.map(_run, names)))


@pytest.mark.parametrize("name", list(oracle_mutants.MUTANTS))
def test_pins_catch_the_planted_mistake(outcomes, name):
    rc, out = outcomes[name]
    assert rc == 1 and (" failed" in out or " error" in out), f"mutant {name}: pins did not fail (exit {rc})\n{out}"


def test_unknown_mutant_is_refused():
    """The plugin refuses a name it does not know, so a renamed mutant cannot pass by planting nothing."""
    env = dict(os.environ, ORACLE_MUTANT="no_such_mistake")
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "tests.oracle_mutants", "-p",
                        "no:cacheprovider", "tests/test_oracle_density.py::test_weights"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode not in (0, 1)
