"""Model parameter sets.

``paper_nesting(i)``: the five Fermi surfaces of Section "Sign-problem-free UV completion"
(nesting parameters v_1 ... v_5), with u = 0, g = 0.7 sqrt(2), c = 3 and dtau = 0.1.
The paper lists nearest-neighbour amplitudes t_{h,x} = t_{v,y} = 1 and, per nesting value,
t~_{v,x} = -t~_{h,y} and mu_x = -mu_y. Reading used here (the paper calls t~ "next-nearest"
yet indexes it by the x and y directions): t~ is the hop of each band along its weak
direction, i.e. t_v for band x and t_h for band y.

``baseline(L, Nt)``: the couplings of the benchmark configurations (t_x = 1 and t_y = 0.5,
swapped for the second band, mu = -0.5, g = 1, r = 0.5, u = 1, c = 3).

Each function returns keyword arguments for ``hmc.Context``.
"""

import math

_NESTING = {  # i: (t~_{v,x} = -t~_{h,y}, mu_x = -mu_y)
    1: (0.45, -0.47),
    2: (0.48, -0.46),
    3: (0.498, -0.44),
    4: (0.505, -0.44),
    5: (0.5085, -0.44),
}


def paper_nesting(i, r=1.26):
    """Couplings for nesting value v_i (i = 1 ... 5); r defaults to the preconditioner study's."""
    tt, mux = _NESTING[i]
    return dict(dtau=0.1, t_h=(1.0, -tt), t_v=(tt, 1.0), mu=(mux, -mux), g=0.7 * math.sqrt(2.0),
                r=r, u=0.0, c=3.0)


def baseline():
    return dict(dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5, u=1.0, c=3.0)
