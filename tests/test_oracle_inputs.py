"""Pins of the seeded input generator (published SplitMix64 outputs, SU(3) properties)."""
import os

import numpy as np

import lqcd_inputs as li

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_splitmix64_published_sequence():
    # SplitMix64 started from state 0: the first outputs are mix64(k * 0x9E3779B97F4A7C15),
    # k = 1, 2, 3; the published values (with their source) are in golden/splitmix64_state0.txt
    with open(os.path.join(GOLDEN, "splitmix64_state0.txt")) as fh:
        want = [int(line, 16) for line in fh if line.strip() and not line.startswith("#")]
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.array([g * np.uint64(k) for k in range(1, len(want) + 1)], dtype=np.uint64)
    out = li._mix64(z)
    assert [int(v) for v in out] == want


def test_counter_mode_is_position_independent():
    a = li.normal(7, 1, 100)
    b = li.normal(7, 1, 60, start=40)
    assert np.array_equal(a[40:], b)
    c = li.normal(7, 1, 33, start=3)
    assert np.array_equal(a[3:36], c)


def test_normal_moments():
    x = li.normal(11, 2, 200000)
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1) < 0.01
    u = li.uniform(11, 2, 0, 100000)
    assert u.min() > 0 and u.max() <= 1


def test_gauge_links_are_su3():
    U = li.gauge_field((2, 2, 2, 4), 0.6, 3)
    m = U.reshape(-1, 3, 3)
    eye = np.einsum("nab,ncb->nac", m, m.conj())
    assert np.abs(eye - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(m) - 1).max() < 1e-14


def test_gauge_chunking_does_not_change_values():
    a = li.gauge_field((2, 2, 2, 4), 0.6, 3)
    b = li.gauge_field((2, 2, 2, 4), 0.6, 3, chunk_sites=5)
    assert np.array_equal(a, b)


def test_eps_zero_gives_unit_links():
    U = li.gauge_field((2, 2, 2, 2), 0.0, 1)
    assert np.abs(U - np.eye(3)).max() < 1e-14


def test_point_source():
    b = li.point_source((4, 4, 4, 4), 2, 1)
    assert b.sum() == 1 and b[0, 0, 0, 0, 2, 1] == 1
