"""CPU checks of the model presets against the nesting parameters the paper prints.

Section "Sign-problem-free UV completion" lists, for five Fermi surfaces, the hopping amplitudes
(t_{h,x} = t_{v,y} = 1, t~_{v,x} = -t~_{h,y}, mu_x = -mu_y) and the nesting parameters
v_1 ~ 0.149, v_2 ~ 0.072, v_3 ~ 0.036, v_4 ~ 0.018, v_5 ~ 0.0092 (v = tan theta, theta the angle
between the Fermi lines of paired hot spots; theta_1 ~ 8.5 degrees). The hot-spot geometry of a
dispersion fixes v, so these printed pairs pin the reading of the "next-nearest-neighbour" t~."""

import math

import pytest

from paper_2204_14241_gb300 import presets

PRINTED = {  # i: (t~_{v,x} = -t~_{h,y}, mu_x = -mu_y, v_i)
    1: (0.45, -0.47, 0.149),
    2: (0.48, -0.46, 0.072),
    3: (0.498, -0.44, 0.036),
    4: (0.505, -0.44, 0.018),
    5: (0.5085, -0.44, 0.0092),
}


def test_nesting_parameter_of_a_known_crossing():
    # band x: Fermi lines kx = const; band y isotropic at mu = 0, shifted by Q: the diamond
    # |kx| + |ky| = pi, whose lines make 45 degrees with them: v = tan 45 = 1
    v = presets.nesting_parameter((1.0, 1.0), (0.0, 1.0), (0.5, 0.0))
    assert v == pytest.approx(1.0, rel=1e-9)


@pytest.mark.parametrize("i", sorted(PRINTED))
def test_printed_nesting_parameters_with_distance_two_hops(i):
    # t~ read as the hop of distance two along each band's weak direction (the amplitudes the
    # paper lists are then the only non-zero ones): every printed v_i to its printed digits
    tt, mux, v_printed = PRINTED[i]
    v = presets.nesting_parameter((1.0, 0.0), (0.0, 1.0), (mux, -mux), t2_h=(0.0, -tt), t2_v=(tt, 0.0))
    assert v == pytest.approx(v_printed, rel=0.01)
    assert math.degrees(math.atan(v)) == pytest.approx(math.degrees(math.atan(v_printed)), abs=0.05)


@pytest.mark.xfail(strict=True, reason="paper_nesting() reads t~ as a nearest-neighbour hop (the operators "
                                       "have no distance-two hops); its Fermi lines cross at ~88 degrees")
@pytest.mark.parametrize("i", sorted(PRINTED))
def test_paper_nesting_presets_reproduce_the_printed_nesting(i):
    p = presets.paper_nesting(i)
    assert presets.nesting_parameter(p["t_h"], p["t_v"], p["mu"]) == pytest.approx(PRINTED[i][2], rel=0.01)
