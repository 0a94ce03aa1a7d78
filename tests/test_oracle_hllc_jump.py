"""The oracle's HLLC flux (Sec. 4, Toro 2009) pinned by the conservation laws.

HLLC replaces the Riemann fan by two constant states U*_L, U*_R between the
outer waves S_L, S_R, separated by a contact moving at S* across which the
pressure is continuous (p*_L = p*_R = P*).  The conservation laws fix
everything else: across each outer wave the Rankine-Hugoniot condition
    F*_K = F_K + S_K (U*_K - U_K)                      (K = L, R)
holds, and across the contact
    F*_R - F*_L = S* (U*_R - U*_L),
with both star states moving at S* and carrying their own side's tangential
velocity.  A star state that moves at S* under pressure P* has the physical
flux F(U*) = S* U* + P* (0, 1, 0, 0, S*), so the flux the solver returns in
the star region is the unique F with F = F_K + S_K (U* - U_K) = F(U*): a
wrong coefficient anywhere in the star state, its energy term included,
breaks it.

Each branch of the solver is reached by a Galilean boost of the same pair of
states (a frame moving at a between the waves): the wave speeds shift by a
and the pressure does not change.  The test reads the star-region flux from
the solver, recovers U*_K from the Rankine-Hugoniot condition, and checks the
remaining conditions in the boosted frame and, after boosting back, the
contact condition in the lab frame.
"""
import numpy as np
import pytest


def euler_state_and_flux(prim, gamma):
    """Conserved state and normal flux of a 1-D face-frame state
    (rho, u, v1, v2, P): written out from the Euler equations."""
    r, u, v1, v2, p = prim
    E = p / (gamma - 1.0) + 0.5 * r * (u * u + v1 * v1 + v2 * v2)
    U = np.array([r, r * u, r * v1, r * v2, E])
    F = np.array([r * u, r * u * u + p, r * u * v1, r * u * v2, (E + p) * u])
    return U, F


def boost(prim, a):
    out = np.array(prim, dtype=float)
    out[1] -= a
    return out


def unboost_state(U, a):
    """A conserved state seen in a frame moving at a along the normal,
    expressed in the lab frame: same density, normal velocity + a."""
    r, m = U[0], U[1]
    return np.array([r, m + r * a, U[2], U[3], U[4] + m * a + 0.5 * r * a * a])


def random_pairs(rng, count):
    out = []
    while len(out) < count:
        L = [rng.uniform(0.1, 10.0), rng.uniform(-3.0, 3.0), rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0),
             rng.uniform(0.05, 20.0)]
        R = [rng.uniform(0.1, 10.0), rng.uniform(-3.0, 3.0), rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0),
             rng.uniform(0.05, 20.0)]
        out.append((np.array(L), np.array(R)))
    return out


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_hllc_satisfies_the_jump_conditions_in_all_four_wave_configurations(oracle, gamma):
    rng = np.random.default_rng(1707)
    checked = {"left": 0, "star_left": 0, "star_right": 0, "right": 0}
    for L, R in random_pairs(rng, 300):
        sl, ss, sr, ps = oracle.star_state(L, R, gamma)
        cl, cr = np.sqrt(gamma * L[4] / L[0]), np.sqrt(gamma * R[4] / R[0])
        # Davis wave speeds, and a contact speed that makes both sides' star
        # pressures equal: p*_L = p_L + rho_L (S_L - u_L)(S* - u_L) = p*_R
        assert sl == min(L[1] - cl, R[1] - cr) and sr == max(L[1] + cl, R[1] + cr)
        assert sl < ss < sr
        pscale = max(L[4], R[4]) + max(L[0] * cl * cl, R[0] * cr * cr) + ps
        psl = L[4] + L[0] * (sl - L[1]) * (ss - L[1])
        psr = R[4] + R[0] * (sr - R[1]) * (ss - R[1])
        assert abs(psl - ps) <= 1e-12 * pscale and abs(psr - ps) <= 1e-12 * pscale
        width = min(ss - sl, sr - ss)
        if width < 0.05 * (sr - sl):
            continue  # a star region too thin to boost into without cancellation
        star = {}
        for name, a in (("left", sl - 0.5), ("star_left", 0.5 * (sl + ss)), ("star_right", 0.5 * (ss + sr)),
                        ("right", sr + 0.5)):
            Lb, Rb = boost(L, a), boost(R, a)
            F = oracle.hllc_1d(Lb, Rb, gamma)
            slb, ssb, srb, psb = oracle.star_state(Lb, Rb, gamma)
            # the boost shifts every wave speed by a and leaves P* alone
            sscale = abs(a) + sr - sl
            assert abs(slb - (sl - a)) <= 1e-13 * sscale and abs(srb - (sr - a)) <= 1e-13 * sscale
            assert abs(ssb - (ss - a)) <= 1e-12 * sscale and abs(psb - ps) <= 1e-11 * pscale
            UL, FL = euler_state_and_flux(Lb, gamma)
            UR, FR = euler_state_and_flux(Rb, gamma)
            fscale = np.abs(FL) + np.abs(FR) + (np.abs(UL) + np.abs(UR)) * sscale + pscale * (1.0 + sscale)
            if name == "left":
                np.testing.assert_allclose(F, FL, rtol=0, atol=1e-13 * fscale.max())
            elif name == "right":
                np.testing.assert_allclose(F, FR, rtol=0, atol=1e-13 * fscale.max())
            else:
                K, (UK, FK, SK, prim) = name[5:], ((UL, FL, slb, Lb) if name == "star_left" else (UR, FR, srb, Rb))
                # U*_K from the Rankine-Hugoniot condition across S_K
                Us = UK + (F - FK) / SK
                assert Us[0] > 0.0
                # it moves with the contact and keeps its side's tangential velocity
                assert abs(Us[1] / Us[0] - ssb) <= 1e-11 * sscale
                assert abs(Us[2] / Us[0] - prim[2]) <= 1e-11 * (1.0 + abs(prim[2]))
                assert abs(Us[3] / Us[0] - prim[3]) <= 1e-11 * (1.0 + abs(prim[3]))
                # and its flux is the physical one at velocity S* and pressure P*
                Fphys = ssb * Us + psb * np.array([0.0, 1.0, 0.0, 0.0, ssb])
                np.testing.assert_allclose(F, Fphys, rtol=0, atol=1e-11 * fscale.max(), err_msg=name)
                star[K] = (unboost_state(Us, a), a)
            checked[name] += 1
        if len(star) == 2:
            # the contact, in the lab frame: F*_R - F*_L = S* (U*_R - U*_L)
            UsL, UsR = star["left"][0], star["right"][0]
            FsL = ss * UsL + ps * np.array([0.0, 1.0, 0.0, 0.0, ss])
            FsR = ss * UsR + ps * np.array([0.0, 1.0, 0.0, 0.0, ss])
            scale = (np.abs(FsL) + np.abs(FsR)).max() + (np.abs(UsL) + np.abs(UsR)).max() * abs(ss)
            np.testing.assert_allclose(FsR - FsL, ss * (UsR - UsL), rtol=0, atol=1e-11 * scale)
            assert UsL[1] / UsL[0] == pytest.approx(ss, abs=1e-11 * (sr - sl))
            assert UsR[1] / UsR[0] == pytest.approx(ss, abs=1e-11 * (sr - sl))
    assert min(checked.values()) >= 100, checked


def test_a_wrong_star_energy_coefficient_breaks_the_jump_conditions(oracle):
    """The check above is sharp: the same recovery applied to a star-region
    flux whose energy component is perturbed by one part in 1e6 of the energy
    scale (a stand-in for a wrong coefficient in the star energy) fails the
    Rankine-Hugoniot / physical-flux consistency."""
    gamma = 1.4
    L = np.array([1.0, 0.3, 0.2, -0.1, 1.0])
    R = np.array([0.125, -0.2, 0.0, 0.4, 0.1])
    sl, ss, sr, ps = oracle.star_state(L, R, gamma)
    a = 0.5 * (sl + ss)
    Lb, Rb = boost(L, a), boost(R, a)
    F = oracle.hllc_1d(Lb, Rb, gamma)
    slb, ssb, _, psb = oracle.star_state(Lb, Rb, gamma)
    UL, FL = euler_state_and_flux(Lb, gamma)
    for eps, ok in ((0.0, True), (1e-6, False)):
        Fp = F.copy()
        Fp[4] += eps * abs(UL[4])
        Us = UL + (Fp - FL) / slb
        Fphys = ssb * Us + psb * np.array([0.0, 1.0, 0.0, 0.0, ssb])
        assert (np.abs(Fp - Fphys).max() <= 1e-11 * np.abs(FL).max()) == ok
