"""Training checkpoint/resume (host logic, no GPU): a run stopped after an
epoch and resumed from its checkpoint takes the same samples in the same
order, with the same step numbers and learning rates, and ends in the same
state as the run that did not stop."""
import numpy as np
import pytest
import torch

from paper_2312_11740_gb300 import learn


class FakeNet:
    """Stands in for the network: Adam-like state updated from the sample,
    step and learning rate, so any change in the order or schedule shows."""

    def __init__(self, n=5):
        self.p = torch.zeros(n, dtype=torch.float32)
        self.m = torch.zeros(n, dtype=torch.float32)
        self.v = torch.zeros(n, dtype=torch.float32)
        self.log = []
        self.cur = None

    def set_loss(self, *a):
        pass

    def set_input2(self, x):
        self.cur = int(x)

    def train_step(self, target, lr, step):
        g = torch.full_like(self.p, float(target)) + self.p
        self.m = 0.9 * self.m + 0.1 * g
        self.v = 0.999 * self.v + 0.001 * g * g
        self.p -= lr * self.m / (self.v.sqrt() + 1e-8)
        self.log.append((self.cur, round(lr, 15), step))
        return float(g.sum())

    def get_params(self):
        return self.p.clone()

    def set_params(self, p):
        self.p = p.clone().float()
        self.m.zero_()
        self.v.zero_()

    def get_adam(self):
        return self.m.clone(), self.v.clone()

    def set_adam(self, m, v):
        self.m, self.v = m.clone().float(), v.clone().float()


def _data(count=7):
    X = np.arange(count)
    Q = np.linspace(-1.0, 1.0, count)
    return X, Q


def test_checkpoint_holds_the_run_state(tmp_path):
    """Checkpointing changes nothing in the run; the file written after the
    last epoch holds its step count, epochs, losses and configuration."""
    X, Q = _data()
    l_ref = learn.train(FakeNet(), X, Q, 3, 1e-2, 11, log=None, lr_final=1e-3, device="cpu")
    ck = str(tmp_path / "ck.npz")
    net = FakeNet()
    l_ck = learn.train(net, X, Q, 3, 1e-2, 11, log=None, lr_final=1e-3, checkpoint=ck,
                       device="cpu")
    assert l_ck == l_ref
    back = FakeNet()
    step, epoch, _, losses, cfg = learn.load_checkpoint(ck, back, device="cpu")
    assert (step, epoch, len(losses)) == (21, 3, 21) and cfg["epochs"] == 3
    assert torch.equal(back.p, net.p) and torch.equal(back.m, net.m)


def test_resume_from_a_middle_epoch_is_bitwise(tmp_path):
    X, Q = _data()
    ref = FakeNet()
    l_ref = learn.train(ref, X, Q, 3, 1e-2, 5, log=None, lr_final=1e-3, device="cpu")
    # the same run, killed after epoch 1: emulate by checkpointing each epoch and
    # keeping the file written after the first one
    ck = str(tmp_path / "ck.npz")
    ck1 = str(tmp_path / "ck1.npz")

    class Stop(Exception):
        pass

    orig = learn.save_checkpoint

    def save_then_stop(path, net, step, epoch, rng, losses, config):
        orig(path, net, step, epoch, rng, losses, config)
        if epoch == 1:
            orig(ck1, net, step, epoch, rng, losses, config)
            raise Stop()

    a = FakeNet()
    learn.save_checkpoint = save_then_stop
    try:
        with pytest.raises(Stop):
            learn.train(a, X, Q, 3, 1e-2, 5, log=None, lr_final=1e-3, checkpoint=ck, device="cpu")
    finally:
        learn.save_checkpoint = orig
    b = FakeNet()
    l_res = learn.train(b, X, Q, 3, 1e-2, 5, log=None, lr_final=1e-3, resume=ck1, device="cpu")
    assert l_res == l_ref
    assert b.log == ref.log[len(X):]  # same samples, steps and learning rates after epoch 1
    assert torch.equal(b.p, ref.p) and torch.equal(b.m, ref.m) and torch.equal(b.v, ref.v)


def test_resume_refuses_another_run(tmp_path):
    X, Q = _data()
    ck = str(tmp_path / "ck.npz")
    learn.train(FakeNet(), X, Q, 1, 1e-2, 5, log=None, checkpoint=ck, device="cpu")
    with pytest.raises(ValueError):
        learn.train(FakeNet(), X, Q, 2, 1e-2, 6, log=None, resume=ck, device="cpu")
