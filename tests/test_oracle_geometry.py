"""Pins of the plan geometry: Eq. n_params, Eq. N_{w'}+W, Eq. N_w, Table 2."""
import math

import numpy as np

from oracle.geometry import (first_tap, fft_size, layers_improved, layers_original,
                             make_geometry, n_minus_one, n_params)


def test_table2_layer_counts(golden):
    # One unknown, dn*dw, fixes row (a) through Eq. N_w; every improved row of
    # Table 2 then follows from Eq. N_{w'}+W (z-offset) or its no-offset form.
    t2 = golden["table2_layers"]
    P = t2["original_a"]["layers"] / (2 * math.pi)
    assert layers_original(P, 1.0) == t2["original_a"]["layers"]
    for row in t2["rows"]:
        got = layers_improved(P, 1.0, row["x0"], row["W"], row["z_offset"])
        assert got == row["layers"], row


def test_gmrt_layer_counts(golden):
    # Section 7: 40 layers without z-offset become 24 with it (W = 7, x0 = 0.25).
    g = golden["gmrt_layers"]
    ok = [P for P in np.linspace(1, 20, 19001)
          if layers_improved(P, 1.0, g["x0"], g["W"], False) == g["no_offset"]]
    assert ok
    assert {layers_improved(P, 1.0, g["x0"], g["W"], True) for P in ok} == {g["offset"]}


def test_n_params_map_sphere_to_pm_z0():
    lmax, z0 = 0.25, 0.25
    ns, n0 = n_params(lmax, lmax, z0, True)
    nmin = math.sqrt(1 - 2 * lmax ** 2)
    assert math.isclose((1 - n0) / ns, z0, rel_tol=1e-14)
    assert math.isclose((nmin - n0) / ns, -z0, rel_tol=1e-12)
    ns2, n02 = n_params(lmax, lmax, z0, False)
    assert n02 == 1.0 and math.isclose((nmin - 1) / ns2, -z0, rel_tol=1e-12)


def test_pixel_z_in_range():
    g = make_geometry(64, 0.25, 7, 0.5, -100, 100)
    z = g.pixel_z()
    assert z.max() <= g.x0 + 1e-15 and z.min() >= -g.x0 - 1e-15
    assert math.isclose(z[32, 32], g.x0, rel_tol=1e-14)        # map centre: n = 1
    assert math.isclose(z[0, 0], -g.x0, rel_tol=1e-12)         # corner: n = n_min


def test_n_minus_one_stable():
    l = np.array([1e-9, 1e-4, 0.3])
    exact = np.sqrt(1 - 2 * l ** 2) - 1
    assert np.allclose(n_minus_one(l, l)[2], exact[2], rtol=1e-14)
    assert math.isclose(n_minus_one(1e-9, 1e-9), -1e-18, rel_tol=1e-12)


def test_fft_size():
    assert fft_size(256, 0.25) == 512
    assert fft_size(2048, 0.25) == 4096
    assert fft_size(1024, 0.25) == 2048
    assert fft_size(4096, 0.375) == 5600          # 4096/0.75 = 5461.3 -> 32 * 175
    assert fft_size(16, 0.25) == 32


def test_first_tap_rule():
    # Section 3.3: nu in [-1/2, 1/2) and the W taps r = first + i are exactly the
    # integers with -W/2 < r - u' <= W/2.
    rng = np.random.default_rng(0)
    for W in (1, 4, 7):
        u = rng.uniform(-50, 50, 1000)
        u[:3] = [0.5, -0.5, 3.0]                         # exact ties
        r0, nu = first_tap(u, W)
        assert nu.min() >= -0.5 and nu.max() < 0.5
        for i in range(W):
            d = r0 + i - u
            assert np.all(d > -W / 2 - 1e-12) and np.all(d <= W / 2 + 1e-12)
            assert np.allclose(d, i - (W - 1) / 2 - nu, atol=1e-12)


def test_plane_range_covers_data_and_obeys_bound():
    for W in (4, 7):
        g = make_geometry(256, 0.25, W, 0.2, -7372.8, 7372.8)
        dn = -n_minus_one(0.1, 0.1)
        assert g.Nw <= layers_improved(dn, 2 * 7372.8, g.x0, W) + 1
        t0, _ = first_tap(np.array([-7372.8, 7372.8]) * g.nscale, W)
        assert t0[0] == g.t_lo and t0[1] + W - 1 == g.t_hi
