"""The oracle's pins catch plausible mistakes: each test plants one mistake in the
oracle (on the CPU, through monkeypatch) and checks that the pin meant to guard that
part now fails.  A pin that still passed would not be pinning anything."""
import numpy as np
import pytest

import test_oracle_contract as TC
import test_oracle_dirac as TD
import test_oracle_force as TF
import test_oracle_hisq as THQ
import test_oracle_multigrid as TM
import test_oracle_ptc as TP
import test_oracle_solvers as TS
from oracle import contract, dirac, force, hisq, multigrid, ptc, solvers
from oracle import lattice as L


def _fails(fn, *args, **kw):
    with pytest.raises(AssertionError):
        fn(*args, **kw)


def test_swapped_hopping_projectors(monkeypatch):
    """(1 + gamma) forward and (1 - gamma) backward instead of the reverse."""
    monkeypatch.setattr(dirac, "GAMMA", -dirac.GAMMA)
    _fails(TD.test_free_field_plane_wave, (1, 0, 2, 1), -1)
    _fails(TD.test_dense_matrix_matches, (2, 2, 2, 2), -1)


def test_dropped_antiperiodic_sign(monkeypatch):
    monkeypatch.setattr(L, "time_boundary_sign", lambda dims, tb, fwd: np.ones(dims[::-1]))
    _fails(TD.test_free_field_plane_wave, (1, 0, 2, 1), -1)


def test_clover_sign(monkeypatch):
    orig = dirac.sigma
    monkeypatch.setattr(dirac, "sigma", lambda mu, nu: -orig(mu, nu))
    _fails(TD.test_clover_abelian_constant_field, 1)


def test_transposed_field_strength(monkeypatch):
    orig = dirac.field_strength
    monkeypatch.setattr(dirac, "field_strength", lambda U, mu, nu: np.swapaxes(orig(U, mu, nu), -1, -2))
    _fails(TD.test_dense_matrix_matches, (4, 2, 2, 4), -1)


def test_missing_trace_subtraction(monkeypatch):
    def no_trace(U, mu, nu):
        q = dirac.clover_leaves(U, mu, nu)
        return (q - dirac._dag(q)) / 8.0

    monkeypatch.setattr(dirac, "field_strength", no_trace)
    _fails(TD.test_clover_abelian_constant_field, 1)


def test_wrong_schur_source_sign(monkeypatch):
    def bad(self, b):
        t = dirac.apply_site_matrix(self.Ainv, b * self.odd)
        return (b - self.kappa * self.H(t)) * self.even

    monkeypatch.setattr(dirac.WilsonClover, "schur_source", bad)
    _fails(TD.test_dense_matrix_matches, (2, 2, 2, 2), -1)


def test_wrong_reconstruction_sign(monkeypatch):
    """x_o = A_oo^-1 (b_o - kappa D_oe x_e) instead of + kappa."""
    def bad(self, xe, b):
        xe = xe * self.even
        xo = dirac.apply_site_matrix(self.Ainv, (b - self.kappa * self.H(xe)) * self.odd) * self.odd
        return xe + xo

    monkeypatch.setattr(dirac.WilsonClover, "reconstruct", bad)
    _fails(TS.test_even_odd_solve_matches_dense, (2, 2, 2, 2), "bicgstab")


def test_anisotropic_weight_on_the_wrong_axis(monkeypatch):
    orig = dirac.anisotropic

    def bad(U, kappa, xi0, nu, csw_t, csw_r, t_boundary=-1):
        op = orig(U, kappa, xi0, nu, csw_t, csw_r, t_boundary)
        w = nu / xi0
        op.hop_weights = (1.0, w, w, w)  # t weighted, x not
        return op

    monkeypatch.setattr(dirac, "anisotropic", bad)
    _fails(TD.test_anisotropic_free_field_plane_wave, (1, 0, 2, 1))


def test_transposed_gamma_in_contraction(monkeypatch):
    orig = contract.contract
    monkeypatch.setattr(contract, "contract",
                        lambda A, B, gamma=None, mom=(0, 0, 0): orig(A, B, None if gamma is None else gamma.T, mom))
    _fails(TC.test_contract_gamma_structure)


def test_momentum_phase_sign(monkeypatch):
    orig = contract.momentum_phase
    monkeypatch.setattr(contract, "momentum_phase", lambda dims, mom: np.conj(orig(dims, mom)))
    import workloads as W
    from _dense_ref import dense_matrix

    U = L.gauge_from_qdp(W.gauge_links(TC.DIMS, 0.4, 5), TC.DIMS)
    op = dirac.WilsonClover(U, TC.KAPPA, TC.CSW)
    Minv = np.linalg.inv(dense_matrix(U, TC.DIMS, TC.KAPPA, TC.CSW))
    _fails(TC.test_wall_source_two_point_eq1_third_line, (U, op, Minv))


def test_multigrid_wrong_chirality_split(monkeypatch):
    """Splitting spins (0, 2) / (1, 3) instead of the gamma_5 eigenspaces."""
    orig = multigrid.chirality_halves

    def bad(internal):
        if internal == (4, 3):
            return (np.s_[0:4:2, :], np.s_[1:4:2, :])
        return orig(internal)

    monkeypatch.setattr(multigrid, "chirality_halves", bad)
    _fails(TM.test_coarse_operator_inherits_gamma5_hermiticity)


def test_transport_without_dagger(monkeypatch):
    monkeypatch.setattr(ptc, "_dag", lambda u: u)
    _fails(TP.test_transport_adjoint)


def test_network_gradient_without_conjugate(monkeypatch):
    """The weight gradient of a layer built from T_s x instead of conj(T_s x)."""
    def bad(U, W, x, g_out, t_boundary=-1):
        cout, cin = W.shape[:2]
        gW = np.zeros_like(W)
        gx = np.zeros_like(x)
        for c in range(cin):
            for s in range(ptc.NSHIFT):
                ts = ptc.transport(U, x[c], s, t_boundary)
                go = g_out.reshape(cout, -1, 4, 3)
                gW[:, c, s] = np.einsum("oxac,xbc->oab", go, ts.reshape(-1, 4, 3))
                back = np.einsum("oba,o...bc->...ac", W[:, c, s].conj(), g_out)
                gx[c] += ptc.transport_adjoint(U, back, s, t_boundary)
        return gW, gx

    monkeypatch.setattr(ptc, "layer_backward", bad)
    _fails(TP.test_gradient_finite_differences, 0)


def test_sequential_source_gamma_on_the_wrong_index(monkeypatch):
    """gamma_5 applied to the source spin of S_0 instead of its sink spin."""
    def bad(S, t, mom=(0, 0, 0), gamma=None):
        gm = contract.G.GAMMA5 if gamma is None else gamma
        dims = (S.shape[3], S.shape[2], S.shape[1], S.shape[0])
        ph = np.conj(contract.momentum_phase(dims, mom))
        X = np.zeros_like(S)
        X[t] = np.einsum("...jkab,kl->...jlab", S[t], gm.T) * ph[t][..., None, None, None, None]
        return X

    monkeypatch.setattr(contract, "sequential_source", bad)
    import workloads as W
    from _dense_ref import dense_matrix

    U = L.gauge_from_qdp(W.gauge_links(TC.DIMS, 0.4, 5), TC.DIMS)
    op = dirac.WilsonClover(U, TC.KAPPA, TC.CSW)
    Minv = np.linalg.inv(dense_matrix(U, TC.DIMS, TC.KAPPA, TC.CSW))
    _fails(TC.test_three_point_eq3_eq4, (U, op, Minv))


def test_restriction_without_conjugate(monkeypatch):
    """P^T v instead of P^+ v."""
    def bad(self, v):
        w = multigrid._blocked(v, self.block)
        out = np.zeros(self.coarse_shape, dtype=np.complex128)
        for chi, h in enumerate(self.halves):
            part = w[(Ellipsis,) + h].reshape(self.coarse_sites + (-1,))
            out[..., chi, :] = np.einsum("...dn,...d->...n", self.basis[chi], part)
        return out

    monkeypatch.setattr(multigrid.Prolongator, "restrict", bad)
    _fails(TM.test_prolongator_orthonormal_and_chiral)


def test_slab_boundary_sign_not_folded(monkeypatch):
    """The slab evaluator without the fermion time-boundary sign on the t links."""
    from oracle import residual

    orig = residual.slab_operator
    monkeypatch.setattr(residual, "slab_operator",
                        lambda g, dims, k, c, t0, t1, tb=-1, hw=None, pc=None: orig(g, dims, k, c, t0, t1, 1, hw, pc))
    _fails(TD.test_slabwise_operator_matches_whole_lattice, (4, 2, 6, 8), 3, -1)


def test_adam_without_bias_correction(monkeypatch):
    def bad(weights, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        state["t"] = state.get("t", 0) + 1
        out = []
        for i, (Wt, g) in enumerate(zip(weights, grads)):
            gr = np.stack([g.real, g.imag])
            m = state.setdefault(("m", i), np.zeros_like(gr))
            v = state.setdefault(("v", i), np.zeros_like(gr))
            m[:] = b1 * m + (1 - b1) * gr
            v[:] = b2 * v + (1 - b2) * gr * gr
            upd = lr * m / (np.sqrt(v) + eps)
            out.append(Wt - (upd[0] + 1j * upd[1]))
        return out

    monkeypatch.setattr(ptc, "adam_step", bad)
    _fails(TP.test_adam_two_steps_closed_form)


def test_adam_second_moment_of_the_wrong_step(monkeypatch):
    """The second moment bias-corrected with b1 instead of b2."""
    orig = ptc.adam_step
    monkeypatch.setattr(ptc, "adam_step", lambda w, g, s, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8:
                        orig(w, g, s, lr=lr, b1=b1, b2=b1, eps=eps))
    _fails(TP.test_adam_two_steps_closed_form)


def test_hisq_seven_staple_coefficient(monkeypatch):
    """1/192 instead of 1/384 for the 7-link staples of the first level."""
    monkeypatch.setattr(hisq, "FAT7", (1 / 8, 1 / 16, 1 / 64, 1 / 192, 0.0))
    _fails(THQ.test_abelian_flux_closed_form, 1)


def test_hisq_lepage_sign(monkeypatch):
    monkeypatch.setattr(hisq, "ASQ", (5 / 8, 1 / 16, 1 / 64, 1 / 384, 1 / 16))
    _fails(THQ.test_abelian_flux_closed_form, 1)


def test_hisq_backward_staple_end_point(monkeypatch):
    """The backward staple closing at U_rho(x - rho) instead of U_rho(x - rho + mu)."""
    orig = hisq.staple

    def bad(U, mu, rho, sign, F):
        if sign > 0:
            return orig(U, mu, rho, sign, F)
        back = hisq._shift(U[rho], rho, -1)
        return hisq._dag(back) @ hisq._shift(F, rho, -1) @ back

    monkeypatch.setattr(hisq, "staple", bad)
    _fails(THQ.test_smearing_gauge_covariance, hisq.FAT7)


def test_hisq_five_staples_one_ordering(monkeypatch):
    """5-link staples summed over one ordering of each pair of directions only."""
    def half_smear(U, coeffs):
        c1, c3, c5, c7, cl = coeffs
        out = np.empty_like(U)
        for mu in range(4):
            perp = [r for r in range(4) if r != mu]
            acc = c1 * U[mu]
            for rho in perp:
                for s in (1, -1):
                    acc = acc + c3 * hisq.staple(U, mu, rho, s, U[mu])
                    for sig in perp:
                        if sig <= rho:
                            continue
                        for s2 in (1, -1):
                            acc = acc + c5 * hisq.staple(U, mu, rho, s, hisq.staple(U, mu, sig, s2, U[mu]))
            out[mu] = acc
        return out

    monkeypatch.setattr(hisq, "smear", half_smear)
    _fails(THQ.test_free_field, 0.0)


def test_hisq_projection_power(monkeypatch):
    """V (V^+ V)^(+1/2) instead of V (V^+ V)^(-1/2)."""
    def bad(V):
        lam, E = np.linalg.eigh(hisq._dag(V) @ V)
        return V @ ((E * np.sqrt(lam)[..., None, :]) @ hisq._dag(E))

    monkeypatch.setattr(hisq, "u3_project", bad)
    _fails(THQ.test_u3_projection_is_the_polar_factor)


def test_hisq_naik_shifted(monkeypatch):
    """Naik link starting one site late: W(x + mu) W(x + 2 mu) W(x + 3 mu)."""
    def bad(Wl):
        out = np.empty_like(Wl)
        for mu in range(4):
            out[mu] = hisq._shift(Wl[mu], mu, 1) @ hisq._shift(Wl[mu], mu, 2) @ hisq._shift(Wl[mu], mu, 3)
        return out

    monkeypatch.setattr(hisq, "naik", bad)
    _fails(THQ.test_naik_link_paths)
    _fails(THQ.test_hisq_links_gauge_covariance)


def test_force_leaf_offset(monkeypatch):
    """Clover force: the third factor of the first leaf credited one site off in mu."""
    bad = list(force.LEAVES)
    bad[0] = (bad[0][0], bad[0][1], (0, True, (1, 1)), bad[0][3])
    monkeypatch.setattr(force, "LEAVES", tuple(bad))
    _fails(TF.test_single_link_variations, -1)


def test_force_odd_trace_without_kappa2(monkeypatch):
    """Clover force: the odd sites' sigma trace without its kappa^2."""
    orig = force.sigma_trace
    calls = []

    def bad(a, b):
        calls.append(1)
        lam = orig(a, b)
        if len(calls) % 2 == 0:  # the second call of each force is the odd pair (W, Z)
            lam = {k: v / (0.12 * 0.12) for k, v in lam.items()}
        return lam

    monkeypatch.setattr(force, "sigma_trace", bad)
    _fails(TF.test_force_is_the_derivative_of_the_action, (2, 2, 2, 2), False)


def test_force_determinant_sign(monkeypatch):
    """Clover force: + 2 log det A_oo instead of - 2 log det A_oo."""
    orig = force.logdet_trace
    monkeypatch.setattr(force, "logdet_trace", lambda ainv: {k: -v for k, v in orig(ainv).items()})
    _fails(TF.test_determinant_term_alone)
