"""Shared pytest configuration.

Markers: ``gpu`` for tests that need a GB300 (they call the CUDA library
through its C ABI); everything else runs on CPU.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libnb")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle():
    from oracle import nb_oracle
    nb_oracle.build()
    return nb_oracle


def _rel_rows(got, ref):
    import numpy as np
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


@pytest.fixture(scope="session")
def trajectory_envelope(oracle):
    """How far the oracle's own shared-step trajectory moves when each of its
    evaluations is perturbed at a given relative level.

    Returns make(m, x, v, eps, h, steps, level, seeds) -> (x_ref, v_ref,
    env_x, env_v): the unperturbed oracle's positions and velocities after
    `steps` shared steps of size h, and per particle the largest relative
    deviation of x and v over runs whose a, jerk and snap carry relative
    perturbations up to `level` (one run per seed).  A path whose evaluations
    agree with the oracle's to `level` may deviate by about that much; close
    pairs that the step resolves poorly amplify any perturbation, and the
    envelope measures by how much.
    """
    import numpy as np

    def make(m, x, v, eps, h, steps, level, seeds=(1, 2)):
        # level: one relative size for a, jerk and snap, or a triple
        ea, ej, es = level if isinstance(level, (tuple, list)) else (level, level, level)
        ref = oracle.Sim(m, x, v, eps=eps, dt_min=h, dt_max=h).init()
        ref.run(steps * h)
        env_x = np.zeros(len(m))
        env_v = np.zeros(len(m))
        for s in seeds:
            o = oracle.Sim(m, x, v, eps=eps, dt_min=h, dt_max=h).set_noise(ea, ej, es, s)
            o.init()
            o.run(steps * h)
            env_x = np.maximum(env_x, _rel_rows(o.x, ref.x))
            env_v = np.maximum(env_v, _rel_rows(o.v, ref.v))
        return ref.x.copy(), ref.v.copy(), env_x, env_v

    return make
