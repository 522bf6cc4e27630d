"""Reference of the online data-collection gate (Sec. 2.2, Algorithm 1) and the
training schedule around it (Sec. 2.3).

TEST INFRASTRUCTURE ONLY.

Readings of the paper used here (it leaves these open or prints them garbled):
* M_p is the unweighted mean of the last p values *including* the current one;
  with fewer than p values, the mean of those available.  p = 10.
* A step is "good" when E_k < M_p(E) and TOS < M_p(TOS); good steps are not
  stored.  Otherwise the (b, x) pair is a candidate.
* The spread check compares solutions x: the candidate is admitted if
  |cos angle(x_n, x_c)| <= theta for every x_c already in C_t (the candidates
  gathered since the last training call).  theta = 0.9.
* During warm-up (steps before tau0) every pair is admitted; the gate only
  runs from step tau0 on.  Warm-up pairs go to the training set X_t, not to
  C_t: Algorithm 1 starts from an empty C_t right after the warm-up training.
* The retraining counter N of Algorithm 1 counts every step after warm-up that
  fails the M_p test, whether or not its pair passes the spread check (the
  algorithm increments N after the spread test, outside it).  Retraining is
  due once N >= f_r; training resets N and empties C_t.
"""

import math

import numpy as np


def moving_average(values, p):
    """M_p over the last p values of ``values`` (which already holds the
    current value as its last entry)."""
    if len(values) == 0:
        raise ValueError("empty history")
    tail = values[-p:]
    return sum(tail) / len(tail)


def is_good(E_hist, T_hist, p):
    """Both criteria of Algorithm 1 for the last entry of each history."""
    return (E_hist[-1] < moving_average(E_hist, p)) and (T_hist[-1] < moving_average(T_hist, p))


def abs_cos(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    na = math.sqrt(float(a @ a))
    nb = math.sqrt(float(b @ b))
    if na == 0.0 or nb == 0.0:
        return 1.0
    return abs(float(a @ b)) / (na * nb)


def spread_ok(x_n, candidates, theta):
    return all(abs_cos(x_n, xc) <= theta for xc in candidates)


class GateRef:
    """Step-by-step decisions of the collection policy.

    ``step(E, TOS, x)`` returns True when the pair is admitted to the replay
    buffer.  ``trained()`` empties C_t and resets N, as after a training call.
    ``N`` is Algorithm 1's count of under-performing steps since then;
    ``due(f_r)`` says whether retraining is due.
    """

    def __init__(self, p=10, theta=0.9, warmup=50):
        self.p = p
        self.theta = theta
        self.warmup = warmup
        self.E = []
        self.T = []
        self.C = []
        self.N = 0
        self.steps = 0

    def step(self, E, TOS, x):
        self.E.append(float(E))
        self.T.append(float(TOS))
        self.steps += 1
        if self.steps <= self.warmup:
            return True
        if is_good(self.E, self.T, self.p):
            return False
        self.N += 1
        if spread_ok(x, self.C, self.theta):
            self.C.append(np.asarray(x, dtype=np.float64))
            return True
        return False

    def trained(self):
        self.C = []
        self.N = 0

    def due(self, f_r):
        return self.N >= f_r
