"""Host logic of the training driver (train.py): the blow-up safeguard restores the
last snapshot in a fresh context and halves the learning rate; repeated blow-ups
end the run.  The solver is a scripted stand-in, so no GPU is needed."""
import numpy as np
import pytest

from paper_2312_11093_gb300 import mgcnn
from paper_2312_11093_gb300 import train as T


class ScriptedSolver:
    """Stands in for mgcnn.Solver: train_step returns the next scripted loss and
    moves the weights by one, so every weight blob records the steps it took."""
    losses = []
    created = []

    def __init__(self, *args, **kwargs):
        self.w = None
        self.lrs = []
        ScriptedSolver.created.append(self)

    def set_weights(self, w):
        self.w = np.array(w, dtype=np.float64)

    def get_weights(self):
        return self.w.copy()

    def train_step(self, problems, K, lr):
        self.lrs.append(lr)
        loss = ScriptedSolver.losses.pop(0)
        if loss == "nonfinite":
            raise mgcnn.MGCNNError(mgcnn.ERR_NONFINITE, "scripted")
        self.w = self.w + 1.0
        return loss

    def close(self):
        pass


@pytest.fixture
def scripted(monkeypatch):
    monkeypatch.setattr(T.mgcnn, "Solver", ScriptedSolver)
    monkeypatch.setattr(T, "make_batch", lambda step, sizes, counts: [])
    ScriptedSolver.created = []
    return ScriptedSolver


def run(losses, steps, max_restarts=8):
    ScriptedSolver.losses = list(losses)
    return T.train(schedule=[((63,), (1,), steps, 1e-3)], init=np.zeros(4), out=None, snapshot_every=5,
                   spike=50.0, max_restarts=max_restarts, log_every=10 ** 9)


def test_nonfinite_loss_restores_the_snapshot_and_halves_the_rate(scripted):
    # steps 0..11 fine, step 12 fails (NaN/Inf in the unrolled cycles), then fine
    w, hist = run([1.0] * 12 + ["nonfinite"] + [1.0] * 7, 20)
    assert len(scripted.created) == 2                      # a fresh context after the failure
    first, second = scripted.created
    assert first.lrs == [1e-3] * 13 and second.lrs == [5e-4] * 7
    # the snapshot was taken at step 10 (after 11 updates): the second context starts there
    assert len(hist) == 19 and all(np.isfinite(hist))
    assert np.array_equal(w, np.full(4, 11.0 + 7.0))


def test_loss_spike_counts_as_a_blow_up(scripted):
    losses = [1.0] * 16 + [1.0e4] + [1.0] * 3                # 1e4 > 50 x the median of the last 20
    w, hist = run(losses, 20)
    assert len(scripted.created) == 2
    assert scripted.created[1].lrs == [5e-4] * 3
    assert 1.0e4 not in hist
    assert np.array_equal(w, np.full(4, 16.0 + 3.0))       # snapshot at step 15 holds 16 updates


def test_repeated_blow_ups_end_the_run(scripted):
    with pytest.raises(RuntimeError):
        run([1.0] * 6 + ["nonfinite"] * 3, 9, max_restarts=2)


def test_paper_batch_is_the_papers_family():
    """make_paper_batch draws the paper's white-noise coefficient as mu = coef h on
    the interior nodes (coef in [1e-3, 1]) with white-noise right-hand sides, per
    size and count, reproducibly per step."""
    probs = T.make_paper_batch(3, sizes=(15, 31), per_size=(2, 1))
    assert [n for _, _, n in probs] == [15, 15, 31]
    for mu, f, n in probs:
        assert mu.shape == (n * n,) and f.shape == (n * n,)
        coef = mu * (n + 1)
        assert coef.min() >= 1e-3 * (1 - 1e-12) and coef.max() <= 1.0
    again = T.make_paper_batch(3, sizes=(15, 31), per_size=(2, 1))
    assert all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) for a, b in zip(probs, again))
    assert not np.array_equal(T.make_paper_batch(4, sizes=(15,), per_size=1)[0][0], probs[0][0])


def test_paper_workload_rejects_divergence_form_hard_modes():
    with pytest.raises(ValueError):
        T.train(schedule=[((15,), (1,), 1, 1e-4)], workload="paper", hard_every=5, out=None)


def test_shipped_paper_weights_fit_the_network():
    """The shipped weights of the paper-family network are one finite blob of the
    8-channel, one-down-one-up layout."""
    w = np.load(T.PAPER_WEIGHTS)
    assert w.dtype == np.float64 and w.shape == (mgcnn.weight_count(8, 1, 1),) and np.isfinite(w).all()
