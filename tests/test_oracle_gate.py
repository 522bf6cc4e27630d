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
