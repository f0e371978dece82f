"""Pins of the oracle's particle reset (Sec. 2.1, Appendix A: particles that leave the
state-variable bounds, or are older than T_max, get new random initial conditions
from their group's box).

* Without bounds and age limit it is the plain integrator.
* With dx/dt = 0 the state only changes at resets, so the reset draws are pinned to
  SplitMix64's published outputs for seed 1234567: the r-th reset of group particle
  j (group of `count`, dim 1) takes output n = r * count + j + 1.
* Ages, reset counts and the check schedule (global step numbers that are multiples
  of check_every) follow from integer arithmetic.
* A harmonic oscillator leaving |x| <= 0.5 is reset at the first check after the
  step at which the closed-form RK4 solution T(hA)^n x0 leaves the box.
"""
import numpy as np

import oracle
from conftest import load_golden

GOLD = load_golden("splitmix64_seed1234567.txt")
OUT = {int(k): int(v[0]) for k, v in GOLD.items()}


def still(count, seed=1234567, lo=0.0, hi=2.0 ** 24):
    return dict(count=count, lo=[lo], hi=[hi], direction=1, seed=seed)


def test_no_reset_is_plain_integration():
    A = np.array([[0.0, 1.0], [-4.0, -0.2]])
    g = dict(count=50, lo=[-1, -1], hi=[1, 1], direction=-1, seed=3)
    x0 = oracle.seed_group(2, g["lo"], g["hi"], g["seed"], count=50)
    got, age, resets = oracle.integrate_reset(oracle.LINEAR, x0, A.reshape(-1), [g], 0.01, 77)
    want = oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), -0.01, 77)
    np.testing.assert_array_equal(got, want)
    assert (age == 77).all() and (resets == 0).all()


def test_age_limit_draws_published_outputs():
    # one particle, dim 1, dx/dt = 0: resets at steps 4, 8, 12 (max_age 4, checked every step)
    g = still(1)
    x0 = np.array([[float(OUT[1] >> 40)]])
    x, age, resets = oracle.integrate_reset(oracle.LINEAR, x0, [0.0], [g], 0.1, 9, max_age=4)
    assert resets[0] == 2 and age[0] == 1
    assert x[0, 0] == float(OUT[3] >> 40)  # second reset: output n = 2 * 1 + 0 + 1
    x, age, resets = oracle.integrate_reset(oracle.LINEAR, x, [0.0], [g], 0.1, 3, step0=9, age=age,
                                            resets=resets, max_age=4)
    assert resets[0] == 3 and age[0] == 0 and x[0, 0] == float(OUT[4] >> 40)


def test_reset_counter_layout_across_particles():
    # group of 2 particles, dim 1: particle j's r-th reset uses output r * 2 + j + 1
    g = still(2)
    x0 = np.array([[float(OUT[1] >> 40), float(OUT[2] >> 40)]])
    x, _, resets = oracle.integrate_reset(oracle.LINEAR, x0, [0.0], [g], 0.1, 2, max_age=1)
    assert list(resets) == [2, 2]
    # r = 2: n = 2*2 + j + 1 = 5 (j=0), 6 (j=1); output 5 is published
    assert x[0, 0] == float(OUT[5] >> 40)


def test_check_schedule_and_bounds():
    g = still(3, seed=11, lo=0.0, hi=1.0)
    x0 = np.array([[0.5, 2.0, np.nan]])  # inside, outside, not finite
    bounds = ([0.0], [1.0])
    x, age, resets = oracle.integrate_reset(oracle.LINEAR, x0, [0.0], [g], 0.1, 2, check_every=3, bounds=bounds)
    assert list(resets) == [0, 0, 0] and list(age) == [2, 2, 2]  # no check yet (global steps 1, 2)
    x, age, resets = oracle.integrate_reset(oracle.LINEAR, x, [0.0], [g], 0.1, 1, step0=2, check_every=3,
                                            bounds=bounds, age=age, resets=resets)
    assert list(resets) == [0, 1, 1] and list(age) == [3, 0, 0]  # checked at global step 3
    assert x[0, 0] == 0.5 and 0.0 <= x[0, 1] < 1.0 and 0.0 <= x[0, 2] < 1.0
    # the new states are the r = 1 draws of particles 1 and 2
    want = oracle.seed_group(1, [0.0], [1.0], 11, idx=[1 * 3 + 1, 1 * 3 + 2])
    assert x[0, 1] == want[0, 0] and x[0, 2] == want[0, 1]


def test_bounds_are_inclusive():
    # a state exactly on a bound is still valid (the box of valid states is closed)
    g = still(2, seed=12, lo=0.0, hi=1.0)
    x0 = np.array([[0.0, 1.0]])
    x, age, resets = oracle.integrate_reset(oracle.LINEAR, x0, [0.0], [g], 0.1, 5, bounds=([0.0], [1.0]))
    assert list(resets) == [0, 0] and list(x[0]) == [0.0, 1.0]
    x, age, resets = oracle.integrate_reset(oracle.LINEAR, np.array([[-1e-6, 1.0 + 2e-7]]), [0.0],
                                            [g], 0.1, 1, bounds=([0.0], [1.0]))
    assert list(resets) == [1, 1]


def test_harmonic_leaves_box_at_closed_form_step():
    w, h = 1.0, 0.01
    A = np.array([[0.0, 1.0], [-w * w, 0.0]])
    Z = h * A
    T = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    x0 = np.array([[0.4], [0.35]])  # amplitude 0.53: leaves |x| <= 0.5
    xs, n_exit = x0.copy(), None
    for n in range(1, 400):
        xs = T @ xs
        if abs(np.float32(xs[0, 0])) > 0.5 or abs(np.float32(xs[1, 0])) > 0.5:
            n_exit = n
            break
    assert n_exit is not None
    g = dict(count=1, lo=[0.0, 0.0], hi=[0.1, 0.1], direction=1, seed=5)
    x, age, resets = oracle.integrate_reset(oracle.HARMONIC, x0, [w], [g], h, n_exit, bounds=([-0.5, -0.5],
                                                                                                [0.5, 0.5]))
    assert resets[0] == 1 and age[0] == 0
    x, age, resets = oracle.integrate_reset(oracle.HARMONIC, x0, [w], [g], h, n_exit - 1,
                                            bounds=([-0.5, -0.5], [0.5, 0.5]))
    assert resets[0] == 0 and age[0] == n_exit - 1
