"""A brute-force, pure-Python restatement of one time step, for tiny grids only.

It differs from the oracle in every structural choice a vectorised implementation can get wrong:
explicit modulo neighbour indexing instead of array rolls, explicit per-link push streaming with
bounce-back (Eq. 3 and Fig. 3 as written, not their pull form), and the collision applied in
velocity space through the dense operator Lambda_bar = M^-1 Lambda M of Eq. 1 with
G = M^-1 S, instead of the moment-space form of Eq. 2.
"""
import numpy as np

from oracle import lattice as L


def _wrap(c, dims):
    return tuple(ci % n for ci, n in zip(c, dims))


def brute_step(f, solid, params):
    """f: (q, *shape) post-streaming state; solid: bool array; params: oracle.lbm.Params."""
    lat = L.lattice(params.lattice)
    q, d = lat.q, lat.d
    shape = solid.shape
    dims = shape[::-1]                       # (nx, ny[, nz])
    nodes = [tuple(reversed(ix)) for ix in np.ndindex(*shape)]   # (x, y[, z]) coordinates

    def at(arr, c):
        return arr[tuple(reversed(_wrap(c, dims)))]

    def plus(c, e):
        return tuple(ci + int(ei) for ci, ei in zip(c, e))

    fluid = lambda c: not bool(at(solid, c))
    rho = {}
    for c in nodes:
        if fluid(c):
            rho[c] = sum(at(f[a], c) for a in range(q))
    # wall nodes and their virtual densities (Eqs. 16-17 with the limiter)
    psi = {}
    eos = params.eos

    def psi_of(r):
        arg = 2.0 * (float(eos.pressure(r)) - r / 3.0) / params.G
        assert arg > 0
        return arg ** 0.5

    for c in nodes:
        if fluid(c):
            psi[c] = psi_of(rho[c])
            continue
        if params.wall == "SF":          # Martys-Chen: no virtual density, psi = 0 on solids
            psi[c] = 0.0
            continue
        num = den = 0.0
        touching = False
        for a in range(1, q):
            nb = plus(c, lat.E[a])
            if fluid(nb):
                touching = True
                num += lat.WF[a] * rho[_wrap(nb, dims)]
                den += lat.WF[a]
        if not touching:
            psi[c] = 0.0
            continue
        if params.wall == "VD":
            rw = params.rho_w_const
        else:
            ra = num / den
            k = float(params.kappa)
            rw = (1 + k) * ra if k >= 0 else ra + k
            rw = min(max(rw, params.rho_g), params.rho_l)
        psi[c] = psi_of(rw)
    lam = np.diag(params.rates())
    LamBar = lat.Minv @ lam @ lat.M
    I = np.eye(q)
    out = np.zeros_like(f)
    tau_e, tau_eps = 1 / params.s_e, 1 / params.s_eps
    for c in nodes:
        if not fluid(c):
            continue
        cc = _wrap(c, dims)
        Fm = np.zeros(d)
        for a in range(1, q):
            Fm += lat.WF[a] * psi[_wrap(plus(c, lat.E[a]), dims)] * lat.E[a]
        Fm = -params.G * psi[cc] * Fm
        F = Fm + np.asarray(params.body_force[:d])
        if params.wall == "SF":          # Eq. 8: adhesion to the solid neighbours
            for a in range(1, q):
                if not fluid(plus(c, lat.E[a])):
                    F = F - params.Gw * rho[cc] * lat.WF[a] * lat.E[a]
        fv = np.array([at(f[a], c) for a in range(q)])
        r = rho[cc]
        u = (lat.E.T.astype(float) @ fv + 0.5 * F) / r
        feq = lat.feq(np.array([r]), u[:, None])[:, 0]
        uF = float(u @ F)
        X = params.sigma * float(Fm @ Fm) / psi[cc] ** 2
        if d == 2:
            S = np.array([0, 6 * uF + 12 * X / (tau_e - 0.5), -6 * uF - 12 * X / (tau_eps - 0.5),
                          F[0], -F[0], F[1], -F[1], 2 * (u[0] * F[0] - u[1] * F[1]), u[0] * F[1] + u[1] * F[0]])
        else:
            S = lat.M @ lat.guo_source(u[:, None], F[:, None])[:, 0]
            S[1] += 114 * X / (tau_e - 0.5)
            S[2] -= 33 * X / (tau_eps - 0.5)
        G = lat.Minv @ S
        fstar = fv - LamBar @ (fv - feq) + (I - 0.5 * LamBar) @ G       # Eq. 1
        # Eq. 3 with halfway bounce-back (push form)
        for a in range(q):
            tgt = plus(c, lat.E[a])
            if fluid(tgt):
                t = _wrap(tgt, dims)
                out[(a,) + tuple(reversed(t))] = fstar[a]
            else:
                out[(lat.OPP[a],) + tuple(reversed(cc))] = fstar[a]
    return out
