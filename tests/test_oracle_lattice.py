"""Pins of the oracle's lattice and collision algebra against facts fixed outside the oracle.

* D2Q9 / D3Q19 isotropy identities of the weights; Eq. 5 force weights give sum w e_x^2 = 1.
* The moment basis is orthogonal (M M^T diagonal) with the textbook row norms.
* m^eq = M f^eq equals the Lallemand-Luo (D2Q9) and d'Humieres (D3Q19) closed forms.
* Eq. 7 with sigma = 0 equals M G for the Guo source written in velocity space.
* With every rate equal and sigma = 0 the MRT collision (Eq. 2) reduces to BGK with Guo forcing,
  written here independently in velocity space.
* The 3D consistency terms give the same per-dimension isotropic pressure-tensor change as Eq. 7.
"""
import numpy as np
import pytest

from oracle import lattice as L, lbm, eos as E


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19], ids=lambda l: l.name)
def test_weight_isotropy(lat):
    E_ = lat.E.astype(float)
    assert abs(lat.W.sum() - 1.0) < 1e-15
    # sum_a w_a e_ai e_aj = c_s^2 delta_ij
    T2 = np.einsum("a,ai,aj->ij", lat.W, E_, E_)
    assert np.allclose(T2, np.eye(lat.d) / 3.0, atol=1e-15)
    # Eq. 5 weights: sum_a w_a e_ai e_aj = delta_ij (so the force is -G psi grad psi to leading order)
    T2f = np.einsum("a,ai,aj->ij", lat.WF, E_, E_)
    assert np.allclose(T2f, np.eye(lat.d), atol=1e-15)
    # fourth-order isotropy of the equilibrium weights: sum w e_x^4 = 3 cs^4, sum w e_x^2 e_y^2 = cs^4
    assert abs(np.sum(lat.W * E_[:, 0] ** 4) - 1.0 / 3.0) < 1e-15
    assert abs(np.sum(lat.W * E_[:, 0] ** 2 * E_[:, 1] ** 2) - 1.0 / 9.0) < 1e-15


def test_d2q9_weights_match_eq5():
    # Eq. 5: w = 1/3 for |e|^2 = 1 and 1/12 for |e|^2 = 2
    n2 = (L.D2Q9.E ** 2).sum(1)
    assert np.all(L.D2Q9.WF[n2 == 1] == 1.0 / 3.0)
    assert np.all(L.D2Q9.WF[n2 == 2] == 1.0 / 12.0)


@pytest.mark.parametrize("lat,norms", [
    (L.D2Q9, [9, 36, 36, 6, 12, 6, 12, 4, 4]),
    (L.D3Q19, [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]),
], ids=["D2Q9", "D3Q19"])
def test_basis_orthogonal(lat, norms):
    G = lat.M @ lat.M.T
    assert np.allclose(G, np.diag(norms), atol=1e-12)
    assert np.allclose(lat.M @ lat.Minv, np.eye(lat.q), atol=1e-13)


def _rand_state(d, n=7, seed=3):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 2.0, n)
    u = rng.uniform(-0.08, 0.08, (d, n))
    F = rng.uniform(-0.01, 0.01, (d, n))
    return rho, u, F


def test_d2q9_meq_closed_form():
    rho, u, _ = _rand_state(2)
    ux, uy = u
    u2 = ux * ux + uy * uy
    meq = L.D2Q9.M @ L.D2Q9.feq(rho, u)
    ref = np.stack([rho, rho * (-2 + 3 * u2), rho * (1 - 3 * u2), rho * ux, -rho * ux, rho * uy, -rho * uy,
                    rho * (ux * ux - uy * uy), rho * ux * uy])
    assert np.allclose(meq, ref, atol=1e-14, rtol=1e-13)


def test_d3q19_meq_closed_form():
    rho, u, _ = _rand_state(3)
    ux, uy, uz = u
    u2 = ux * ux + uy * uy + uz * uz
    meq = L.D3Q19.M @ L.D3Q19.feq(rho, u)
    p3xx = rho * (3 * ux * ux - u2)
    pww = rho * (uy * uy - uz * uz)
    ref = np.stack([rho, -11 * rho + 19 * rho * u2, 3 * rho - 5.5 * rho * u2,
                    rho * ux, -2 / 3 * rho * ux, rho * uy, -2 / 3 * rho * uy, rho * uz, -2 / 3 * rho * uz,
                    p3xx, -0.5 * p3xx, pww, -0.5 * pww,
                    rho * ux * uy, rho * uy * uz, rho * ux * uz,
                    0 * rho, 0 * rho, 0 * rho])
    assert np.allclose(meq, ref, atol=1e-14, rtol=1e-12)


def test_eq7_without_sigma_is_guo_source():
    rho, u, F = _rand_state(2)
    p = lbm.Params("D2Q9", E.cs_config(), sigma=0.0)
    S = lbm.source_moments(p, u, F, F, np.ones_like(rho))
    SG = L.D2Q9.M @ L.D2Q9.guo_source(u, F)
    assert np.allclose(S, SG, atol=1e-15)


def test_d3q19_guo_source_moments():
    # Guo source moments: zero mass, momentum F, and the second-order part u F + F u
    rho, u, F = _rand_state(3)
    G = L.D3Q19.guo_source(u, F)
    E_ = L.D3Q19.E.astype(float)
    assert np.allclose(G.sum(0), 0, atol=1e-16)
    assert np.allclose(np.einsum("ai,an->in", E_, G), F, atol=1e-16)
    P = np.einsum("ai,aj,an->ijn", E_, E_, G)
    ref = np.einsum("in,jn->ijn", u, F) + np.einsum("in,jn->ijn", F, u)
    assert np.allclose(P, ref, atol=1e-16)


def _bgk_guo(f, rho, u, F, s, lat):
    """BGK with Guo forcing in velocity space: f* = f - s (f - f^eq) + (1 - s/2) G."""
    return f - s * (f - lat.feq(rho, u)) + (1 - s / 2) * lat.guo_source(u, F)


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_mrt_reduces_to_bgk(name):
    lat = L.lattice(name)
    shape = (5, 6) if lat.d == 2 else (3, 4, 5)
    rng = np.random.default_rng(11)
    rho0 = rng.uniform(0.2, 0.4, shape)
    u0 = rng.uniform(-0.02, 0.02, (lat.d,) + shape)
    f = lat.feq(rho0, u0) * (1 + 0.01 * rng.uniform(-1, 1, (lat.q,) + shape))
    s = 1.3
    eos = E.cs_config().at_reduced_temperature(0.7)
    p = lbm.Params(name, eos, sigma=0.0, s_rho=s, s_e=s, s_eps=s, s_j=s, s_q=s, s_nu=s, s_pi=s, s_m=s,
                   rho_l=1.0, rho_g=0.001)
    geo = lbm.Geometry(np.zeros(shape, np.uint8), name)
    fstar, (rho, psi, Fm, F, u) = lbm.collide(f, geo, p)
    ref = _bgk_guo(f, rho, u, F, s, lat)
    assert np.max(np.abs(fstar - ref)) < 1e-14


def test_sigma_terms_same_pressure_correction_2d_3d():
    """The consistency source changes the post-collision second moment isotropically; per dimension
    the change must be the same in 2D (Eq. 7) and in the 3D reading."""
    X = 0.37                      # sigma |F_m|^2 / psi^2 with sigma = 1, |F_m| = sqrt(X), psi = 1
    out = {}
    for name in ("D2Q9", "D3Q19"):
        lat = L.lattice(name)
        p = lbm.Params(name, E.cs_config(), sigma=1.0, s_e=0.7, s_eps=1.3)
        d = lat.d
        u = np.zeros((d, 1))
        F = np.zeros((d, 1))
        Fm = np.zeros((d, 1))
        Fm[0] = np.sqrt(X)
        S = lbm.source_moments(p, u, F, Fm, np.ones(1))
        lam = p.rates()[:, None]
        dm = (1 - lam / 2) * S                    # post-collision moment change from S (Eq. 2)
        df = lat.Minv @ dm
        Pi = np.einsum("ai,aj,a->ij", lat.E.astype(float), lat.E.astype(float), df[:, 0])
        assert np.allclose(Pi, Pi[0, 0] * np.eye(d), atol=1e-14)
        out[name] = Pi[0, 0]
    assert abs(out["D2Q9"] - out["D3Q19"]) < 1e-13
    # and in 2D this equals 2 s_e sigma X (Eq. 7: (1 - s_e/2) * 12 sigma X/(tau_e - 1/2) / 3 / 2)
    assert abs(out["D2Q9"] - 2 * 0.7 * X) < 1e-13
