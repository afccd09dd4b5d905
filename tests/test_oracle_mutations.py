"""The model pins catch plausible mistakes in the oracle.

Each case plants one mistake into a private copy of ``oracle/bpf.py`` (on the
CPU, never in the oracle itself): a flipped sign, a dropped square, a
transposed factor.  The copy is loaded as a separate module and the pins of
``test_oracle_model_pins`` that cover the mutated function must fail on it.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

import oracle
from test_oracle_model_pins import CHECKS

HERE = os.path.dirname(os.path.abspath(__file__))
BPF_SRC = os.path.join(os.path.dirname(HERE), "oracle", "bpf.py")

# (name, original text, mutated text, pins that must catch it)
MUTATIONS = [
    ("sv_obs_sign", "s = -0.5 * xx - yy * yy", "s = 0.5 * xx - yy * yy", ["sv_obs"]),
    ("sv_obs_beta_square", "np.exp(-xx) / (2.0 * model.beta ** 2)", "np.exp(-xx) / (2.0 * model.beta)", ["sv_obs"]),
    ("sv_obs_const", "c = -0.5 * np.log(2 * np.pi * model.beta ** 2)", "c = -0.5 * np.log(2 * np.pi * model.beta)",
     ["sv_obs"]),
    ("lg_obs_Lr_transposed", "np.linalg.solve(model.Lr, resid.T)", "np.linalg.solve(model.Lr.T, resid.T)", ["lg_obs"]),
    ("lg_obs_const_dy", "- 0.5 * model.dy * np.log(2 * np.pi)", "- 0.5 * np.log(2 * np.pi)", ["lg_obs"]),
    ("lg_obs_half", "s = -0.5 * np.sum(z * z, axis=1)", "s = -np.sum(z * z, axis=1)", ["lg_obs"]),
    ("mutate_Lq_transposed", "eps @ model.Lq.T", "eps @ model.Lq", ["mutate"]),
    ("mutate_A_transposed", "return xhat @ model.A.T +", "return xhat @ model.A +", ["mutate"]),
    ("mutate_sv_sigma_square", "model.phi * xhat + model.sigma * eps", "model.phi * xhat + model.sigma ** 2 * eps",
     ["mutate_sv"]),
    ("init_L0_transposed", "eps @ model.L0.T", "eps @ model.L0", ["init_lg"]),
    ("init_m0_dropped", "return model.m0[None, :] + eps", "return 0.0 * model.m0[None, :] + eps", ["init_lg"]),
    ("init_sv_variance", "sd0 = model.sigma / np.sqrt(1.0 - model.phi ** 2)", "sd0 = model.sigma / (1.0 - model.phi ** 2)",
     ["init_sv"]),
]


def _mutant(name, old, new):
    src = open(BPF_SRC).read()
    assert src.count(old) == 1, f"mutation {name}: text not found exactly once"
    mod_name = f"oracle._bpf_mutant_{name}"
    spec = importlib.util.spec_from_loader(mod_name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    sys.modules[mod_name] = mod
    try:
        exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod_name]
    return mod


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, pins):
    mut = _mutant(name, old, new)
    for pin in pins:
        with pytest.raises(AssertionError):
            CHECKS[pin](mut)


def test_unmutated_copy_passes():
    """The copying machinery itself does not break the oracle."""
    mod = _mutant("identity", "def obs_terms(", "def obs_terms(")
    for check in CHECKS.values():
        check(mod)
