"""The GPU's HLLC star state is written with the factor (S_K - u_K) cancelled
analytically; this checks, on the host in FP64, that it is the printed form
(Toro's HLLC star state, Sec. 4) to rounding wherever the printed form is
finite, and that it stays finite where S_K = u_K exactly."""
import numpy as np


def star_energy_printed(rho, u, P, E, sk, ss):
    f = rho * (sk - u) / (sk - ss)
    return f * (E / rho + (ss - u) * (ss + P / (rho * (sk - u))))


def star_energy_cancelled(rho, u, P, E, sk, ss):
    rb = 1.0 / (sk - ss)
    f = rho * (sk - u) * rb
    du = ss - u
    return f * (E / rho + du * ss) + du * P * rb


def test_cancelled_form_equals_the_printed_one():
    rng = np.random.default_rng(7)
    n = 200000
    rho = rng.uniform(0.1, 10.0, n)
    u = rng.normal(0.0, 2.0, n)
    P = rng.uniform(0.1, 10.0, n)
    c = np.sqrt(5.0 / 3.0 * P / rho)
    E = P / (2.0 / 3.0) + 0.5 * rho * u * u
    sk = u - c * rng.uniform(1.0, 3.0, n)          # a left wave: S_K < u_K
    ss = u + c * rng.uniform(-0.9, 3.0, n)          # the contact right of it
    a = star_energy_printed(rho, u, P, E, sk, ss)
    b = star_energy_cancelled(rho, u, P, E, sk, ss)
    scale = np.abs(E) + np.abs(rho * (ss - u) * ss) + np.abs(P) + np.abs(a)
    assert np.max(np.abs(a - b) / scale) < 1e-13


def test_cancelled_form_is_finite_where_the_wave_speed_equals_the_flow_speed():
    rho, u, P, E, ss = (np.float64(x) for x in (1.0, 1.0e8, 1e-10, 5e15, 2.0e8))
    sk = u  # a sound speed below the ulp of u: S_K rounds to u_K
    with np.errstate(divide="ignore", invalid="ignore"):
        assert not np.isfinite(star_energy_printed(rho, u, P, E, sk, ss))
    v = star_energy_cancelled(rho, u, P, E, sk, ss)
    # f = 0 there, so the star energy flux term is the pressure work alone
    assert np.isfinite(v) and v == (ss - u) * P / (sk - ss)
