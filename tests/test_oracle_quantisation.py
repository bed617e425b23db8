"""The oracle's quantisation: centres and radii to 1/1024 A, rounded half to even.

The method works on inputs quantised to 2^-10 A. How a value halfway between
two quanta rounds is a reading (round half to even, the IEEE default). These
pins fix it through quantities the definition gives in closed form:

* one ball alone is a vertex of K_alpha with Size -r^2, so the vertex value
  is -R^2 / 2^20 with R the quantised radius;
* two equal balls of radius r whose centres are d quanta apart form an
  unattached edge with Size d^2/4 - r^2. At alpha = 0 the edge is present
  exactly when d <= 2R (AC3 is inclusive). A centre half a quantum beyond
  2R rounds onto 2R under half-to-even, which gives Size exactly 0 and the
  edge, and one quantum further under half-away-from-zero, which loses it.
"""
import numpy as np
import pytest

import oracle

Q = 1024.0

# radius -> quantised radius R = 1024 r rounded half to even
RADII = [
    (1.7, 1741),           # carbon, van der Waals: 1740.8
    (1.55, 1587),          # nitrogen: 1587.2
    (1.52, 1556),          # oxygen: 1556.48
    (1.8, 1843),           # sulphur: 1843.2
    (1.7 + 1.4, 3174),     # carbon + probe: 3174.4
    (1.55 + 1.4, 3021),    # 3020.8
    (1.52 + 1.4, 2990),    # 2990.08
    (1.8 + 1.4, 3277),     # 3276.8
    (1000.5 / Q, 1000),    # halfway, rounds to the even neighbour below
    (1001.5 / Q, 1002),    # halfway, rounds to the even neighbour above
]


@pytest.mark.parametrize("r,R", RADII)
def test_single_ball_vertex_size(r, R):
    res = oracle.alpha_complex(np.array([[0.25, -3.5, 7.0]]), np.array([r]), 0.0)
    assert [len(s) for s in res.simplices] == [1, 0, 0, 0]
    assert not res.attached[0][0]
    assert res.f[0][0] == -(R * R) / 2.0**20


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_halfway_centre_rounds_to_even(sign, axis):
    # equal balls of 1024 quanta; the second centre 2048.5 quanta away rounds to 2048 (even)
    c = np.zeros((2, 3))
    c[1, axis] = sign * 2048.5 / Q
    r = np.array([1.0, 1.0])
    res = oracle.alpha_complex(c, r, 0.0)
    assert res.simplices[1].tolist() == [[0, 1]]
    assert res.f[1][0] == 0.0  # d^2/4 - r^2 = 1024^2 - 1024^2
    assert not res.attached[1][0]


def test_halfway_centre_rounding_up_to_even_loses_the_edge():
    # 2049.5 quanta rounds to 2050: d^2/4 - r^2 = (1025^2 - 1024^2) / 2^20 > 0 = alpha
    c = np.array([[0.0, 0.0, 0.0], [2049.5 / Q, 0.0, 0.0]])
    res = oracle.alpha_complex(c, np.array([1.0, 1.0]), 0.0)
    assert len(res.simplices[1]) == 0
    assert [len(s) for s in res.simplices] == [2, 0, 0, 0]
    # at alpha = that Size the edge is back, with that value
    size = (1025**2 - 1024**2) / 2.0**20
    res = oracle.alpha_complex(c, np.array([1.0, 1.0]), size)
    assert res.simplices[1].tolist() == [[0, 1]]
    assert res.f[1][0] == size


@pytest.mark.parametrize("a_half,present", [(2048.5, False), (2049.5, True), (2050.5, True)])
def test_halfway_alpha_rounds_to_even(a_half, present):
    # equal balls 2050 quanta apart: edge Size (1025^2 - 1024^2) / 2^20 = 2049 / 2^20.
    # alpha = a_half / 2^20: 2048.5 rounds to 2048 (edge absent); 2049.5 and 2050.5 round to 2050 (present).
    c = np.array([[0.0, 0.0, 0.0], [2050.0 / Q, 0.0, 0.0]])
    res = oracle.alpha_complex(c, np.array([1.0, 1.0]), a_half / 2.0**20)
    assert (res.simplices[1].tolist() == [[0, 1]]) == present
    if present:
        assert res.f[1][0] == 2049.0 / 2.0**20
