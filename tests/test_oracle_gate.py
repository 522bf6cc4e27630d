"""Pins of Algorithm 1's gate (Sec. 2.2) on a hand-worked sequence."""
import json
import os

import numpy as np

from oracle import gate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gate_sequence.json")


def test_moving_average_reading():
    assert gate.moving_average([1.0, 2.0, 3.0, 4.0], 3) == 3.0
    assert gate.moving_average([5.0], 10) == 5.0


def test_hand_worked_sequence():
    spec = json.load(open(GOLDEN))
    P = spec["params"]
    g = gate.GateRef(p=P["p"], theta=P["theta"], warmup=P["warmup"])
    for i, s in enumerate(spec["steps"]):
        if s["train_before"]:
            g.trained()
        assert g.step(s["E"], s["TOS"], np.array(s["x"], dtype=float)) == s["admit"], (i, s["why"])


def test_retraining_counter_sequence():
    """Algorithm 1's N: every post-warm-up step that is not good counts, admitted
    or not; a training call resets it (hand-worked column of the golden file)."""
    spec = json.load(open(GOLDEN))
    P = spec["params"]
    g = gate.GateRef(p=P["p"], theta=P["theta"], warmup=P["warmup"])
    for i, s in enumerate(spec["steps"]):
        if s["train_before"]:
            g.trained()
        g.step(s["E"], s["TOS"], np.array(s["x"], dtype=float))
        assert g.N == s["N"], (i, g.N, s["N"])
    assert g.due(3) and not g.due(4)


def test_warmup_pairs_are_not_candidates():
    """The spread check of the first post-warm-up candidate runs against an
    empty C_t, even when a warm-up pair is parallel to it."""
    g = gate.GateRef(p=2, theta=0.9, warmup=2)
    x = np.array([1.0, 0.0])
    assert g.step(1.0, 1.0, x) and g.step(1.0, 1.0, x)
    assert g.step(2.0, 2.0, x)          # not good, C_t empty: admitted
    assert not g.step(3.0, 3.0, x)      # not good, parallel to the admitted one
    assert g.N == 2
