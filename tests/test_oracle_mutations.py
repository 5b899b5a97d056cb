"""The pins of the symmetric variant and of CG / MINRES are not vacuous: a
plausible mistake planted in a copy of the oracle's source (CPU only, nothing
on disk changes) makes at least one pin fail."""
import inspect
import types

import pytest

import oracle.krylov
import oracle.mgcnn
from tests import test_oracle_symmetric as pins


def mutant(module, old: str, new: str):
    """A fresh copy of `module` with one source edit."""
    src = inspect.getsource(module)
    assert src.count(old) == 1, old
    m = types.ModuleType(module.__name__)
    m.__dict__.update(__package__=module.__package__, __file__=module.__file__)
    exec(compile(src.replace(old, new), module.__file__, "exec"), m.__dict__)
    return m


MGCNN_MUTATIONS = {
    "adjoint kernel not flipped": ("W.transpose(1, 0, 2, 3)[:, :, ::-1, ::-1]", "W.transpose(1, 0, 2, 3)"),
    "adjoint kernel not transposed": ("W.transpose(1, 0, 2, 3)[:, :, ::-1, ::-1]", "W[:, :, ::-1, ::-1]"),
    "setup tensor before the adjoint conv": (
        "x[l] = x[l] + s[l] * cn.conv_same_adjoint(x[l], Kd[i])",
        "x[l] = x[l] + cn.conv_same_adjoint(s[l] * x[l], Kd[i])"),
    "up layers in the down order": ("for i in reversed(range(nu)):\n            x[l] = x[l] + s[l]",
                                    "for i in range(nu):\n            x[l] = x[l] + s[l]"),
    "TCNN not tied to RCNN": ("x[l - 1] = x[l - 1] + cn.tcnn(x[l], weights[\"w_R\"], sizes[l - 1])",
                              "x[l - 1] = x[l - 1] + cn.tcnn(x[l], weights[\"w_P\"], sizes[l - 1])"),
    "BPX level weight 2^l": ("np.sqrt(omega * 4.0 ** lev / st.aC)", "np.sqrt(omega * 2.0 ** lev / st.aC)"),
}

KRYLOV_MUTATIONS = {
    "CG beta inverted": ("z + (rz_new / rz) * p", "z + (rz / rz_new) * p"),
    "CG alpha from the wrong product": ("alpha = rz / np.vdot(p, q)", "alpha = rz / np.vdot(q, q)"),
    "MINRES rotation sign": ("delta = cs * dbar + sn * alpha", "delta = cs * dbar - sn * alpha"),
    "MINRES stale epsilon": ("w = (v - eps_old * w_prev2 - delta * w_prev) / gamma",
                             "w = (v - eps * w_prev2 - delta * w_prev) / gamma"),
    "MINRES Lanczos term dropped": ("t = t - (alpha / beta) * r_cur", "t = t - 0.0 * r_cur"),
}


def run_pins():
    """Every symmetric-variant and Krylov pin, each at one parameter set."""
    pins.test_symmetric_network_is_symmetric_and_positive_definite(4, 2)
    pins.test_symmetric_network_equals_general_form_for_uniform_setup()
    pins.test_bpx_network_is_the_textbook_bpx_operator(0.7, 2)
    for k in (2, 4):
        pins.test_pcg_iterate_minimises_the_energy_error(k)
        pins.test_minres_iterate_minimises_the_preconditioned_residual(k)
    pins.test_pcg_identity_preconditioner_solves_the_system()
    pins.test_minres_without_preconditioner_is_minimal_residual()


def test_unmutated_oracle_passes_the_pins():
    run_pins()


@pytest.mark.parametrize("name", list(MGCNN_MUTATIONS))
def test_network_mutation_is_caught(monkeypatch, name):
    monkeypatch.setattr(pins, "omg", mutant(oracle.mgcnn, *MGCNN_MUTATIONS[name]))
    with pytest.raises(AssertionError):
        run_pins()


@pytest.mark.parametrize("name", list(KRYLOV_MUTATIONS))
def test_krylov_mutation_is_caught(monkeypatch, name):
    monkeypatch.setattr(pins, "ok", mutant(oracle.krylov, *KRYLOV_MUTATIONS[name]))
    with pytest.raises(AssertionError):
        run_pins()
