"""Planted mistakes: each one, planted in the oracle on the CPU, fails the pin
that is meant to catch it.

The pins of test_oracle_dg.py check the oracle against closed forms and
invariants.  These controls show that plausible slips in the flux, the
wave-speed bound or the sources do not pass them:

* the pressure term p' of the momentum flux dropped: the flux Jacobian of
  a frozen ideal-gas mixture no longer has spectral radius Lambda (Eq. (3.4));
* the sound speed missing from Lambda: Lambda no longer bounds it;
* the sign of the gravity work in the energy source flipped: E + rho g z is
  no longer conserved (Eq. (2.11e));
* the momentum carried by falling rain dropped (Eq. (2.1e)): the vertical
  momentum flux no longer differs from the no-fall flux by u times the rain
  mass flux.

and for the thermodynamics of test_oracle_thermo.py:

* the exponent a = (c_pv - c_l)/R_v of Eq. (2.6) with the wrong sign:
  e_s no longer solves Clausius-Clapeyron with the linear latent heat;
* the cloud water's heat capacity dropped from the split's energy residual
  (Eq. (2.8a)): the split no longer reproduces the internal energy.

and for the stabilisation of test_oracle_stabilisation.py (Section 3.5-3.6):

* the sponge without its mass fix (the moisture removed not returned to
  rho_d'): the density at a node is no longer kept;
* the interior-penalty term lost (sigma -> 0 inside the form): the SIP
  form is no longer positive semidefinite at sigma = 10;
* the diffusion scaled by a wrong factor: its energy no longer converges to
  alpha int |grad u|^2.

and for the complex-step tangent that the adjoint's tests compare with:

* |x| taken as the complex modulus (np.abs) instead of by the sign of the
  real part: the imaginary part is lost and the tangent no longer matches
  central differences.

A further control, the forward-Euler step planted in place of SSPRK(4,3),
sits beside its pin in test_oracle_dg.py.
"""
import numpy as np
import pytest

from oracle import dg, thermo
from oracle import stabilisation as st
from tests import test_oracle_dg as pins
from tests import test_oracle_stabilisation as stab_pins
from tests import test_oracle_thermo as thermo_pins


def test_dropped_pressure_flux_fails_the_spectral_radius_pin(monkeypatch):
    orig = dg.physical_flux

    def planted(prob, j, P):
        F = orig(prob, j, P)
        F[prob.i_m[j]] = F[prob.i_m[j]] - P["p_prime"]
        return F

    monkeypatch.setattr(dg, "physical_flux", planted)
    with pytest.raises(AssertionError):
        pins.test_lambda_bounds_flux_jacobian_eigenvalues("dry", 0)


def test_lambda_without_sound_speed_fails_the_bound_pin(monkeypatch):
    def planted(prob, j, P):
        lam = np.abs(P["u"][j])
        if j == prob.mesh.vert:
            lam = lam + np.abs(P["v_r"])
        return lam

    monkeypatch.setattr(dg, "wave_speed", planted)
    with pytest.raises(AssertionError):
        pins.test_lambda_bounds_flux_jacobian_eigenvalues("moist_sat", 1)


def test_flipped_gravity_work_fails_the_energy_pin(monkeypatch):
    orig = dg.source

    def planted(prob, Uf, P):
        G = orig(prob, Uf, P)
        G[prob.i_E] = -G[prob.i_E]
        return G

    monkeypatch.setattr(dg, "source", planted)
    with pytest.raises(AssertionError):
        pins.test_total_energy_with_potential_energy_conserved()


def test_dropped_rain_momentum_fails_the_rain_flux_pin(monkeypatch):
    orig = dg.physical_flux

    def planted(prob, j, P):
        F = orig(prob, j, P)
        if j == prob.mesh.vert:
            rvr = P["rho_r"] * P["v_r"]
            for i in range(prob.mesh.dim):
                F[prob.i_m[i]] = F[prob.i_m[i]] + rvr * P["u"][i]
        return F

    monkeypatch.setattr(dg, "physical_flux", planted)
    with pytest.raises(AssertionError):
        pins.test_rain_fluxes_carry_their_energy_and_momentum()


def test_wrong_sign_of_es_exponent_fails_clausius_clapeyron(monkeypatch):
    monkeypatch.setattr(thermo, "ES_A", -thermo.ES_A)
    with pytest.raises(AssertionError):
        thermo_pins.test_es_satisfies_clausius_clapeyron(290.0)


def test_split_without_cloud_heat_capacity_fails_the_invariants(monkeypatch):
    def planted(T, rho_d, rho_m, rho_r, rho_e, rho_v):
        return thermo.internal_energy(rho_d, rho_v, 0.0 * rho_m, rho_r, T) - rho_e

    monkeypatch.setattr(thermo, "_residual", planted)
    with pytest.raises(AssertionError):
        thermo_pins.test_split_invariants()


def test_sponge_without_mass_fix_fails_the_sponge_pin(monkeypatch):
    orig = st.apply_sponge

    def planted(prob, U, z_d, alpha_s):
        V = orig(prob, U, z_d, alpha_s)
        V[prob.i_rd] = U[prob.i_rd]
        return V

    monkeypatch.setattr(st, "apply_sponge", planted)
    with pytest.raises(AssertionError):
        stab_pins.test_sponge_mass_fix_and_damping()


def test_lost_penalty_fails_the_definiteness_pin(monkeypatch):
    orig = st.diffusion_rhs
    monkeypatch.setattr(st, "diffusion_rhs",
                        lambda prob, U, aU, aR, sigma: orig(prob, U, aU, aR, 0.0))
    with pytest.raises(AssertionError):
        stab_pins.test_sip_matrix_symmetric_nullspace_and_definite(2, (True, False))


def test_wrongly_scaled_diffusion_fails_the_laplacian_pin(monkeypatch):
    orig = st.diffusion_rhs
    monkeypatch.setattr(st, "diffusion_rhs",
                        lambda prob, U, aU, aR, sigma: 2.0 * orig(prob, U, aU, aR, sigma))
    with pytest.raises(AssertionError):
        stab_pins.test_sip_converges_to_laplacian()


def test_modulus_for_abs_fails_the_complex_step_pin(monkeypatch):
    monkeypatch.setattr(dg, "_abs", np.abs)
    with pytest.raises(AssertionError):
        pins.test_complex_step_tangent_matches_central_differences()


def test_fallout_with_a_wrong_face_jacobian_fails_the_water_budget_pin(monkeypatch):
    """The wall outflow integrated with the element Jacobian |K|/2^d instead
    of the face's |F|/2^(d-1) (a factor h_j/2 off): the water in the domain
    plus the fall-out is no longer constant."""
    orig = dg.rhs

    def planted(prob, U, elements=None, return_stats=False):
        out = orig(prob, U, elements, return_stats)
        if return_stats:
            R, stats = out
            stats = dict(stats, wall_water_outflow=stats["wall_water_outflow"] * prob.mesh.h[-1] / 2.0)
            return R, stats
        return out

    monkeypatch.setattr(dg, "rhs", planted)
    with pytest.raises(AssertionError):
        pins.test_water_budget_closes_with_the_fallout()


def test_fallout_advanced_by_the_stage_weights_fails_the_water_budget_pin(monkeypatch):
    """The fall-out accumulated with the stage weights of the Shu-Osher form
    (dt/2, dt/2, dt/6, dt/2 on the four outflows) instead of their weights in
    u^{n+1} once the stages are expanded: the budget no longer closes."""
    def planted(prob, U, dt, nsteps, fallout=0.0):
        F = float(fallout)
        for _ in range(nsteps):
            stages = []
            def L(V):
                R, st = dg.rhs(prob, V, return_stats=True)
                stages.append(st["wall_water_outflow"])
                return R
            U = dg.ssprk43_step(L, U, dt)
            F += dt * (0.5 * stages[0] + 0.5 * stages[1] + stages[2] / 6.0 + 0.5 * stages[3])
        return U, F

    monkeypatch.setattr(dg, "run_with_fallout", planted)
    with pytest.raises(AssertionError):
        pins.test_water_budget_closes_with_the_fallout()


def test_flipped_evaporation_temperature_term_fails_its_pin(monkeypatch):
    """The temperature term of the evaporation coefficient of Eq. (2.4) with
    the wrong sign: the coefficient no longer vanishes at 314.17 K."""
    from oracle import constants as C
    monkeypatch.setattr(C, "S_EV_B", -C.S_EV_B)
    with pytest.raises(AssertionError):
        thermo_pins.test_evaporation_coefficient_vanishes_where_the_paper_puts_it()


def test_sound_speed_without_gamma_fails_the_wave_speed_pin(monkeypatch):
    """c = sqrt(p / rho) (gamma dropped): the hand value of the largest wave
    speed at a uniform state no longer matches."""
    monkeypatch.setattr(thermo, "gamma_moist", lambda *a: 1.0)
    with pytest.raises(AssertionError):
        pins.test_max_wave_speed_and_cfl_step_by_hand()
