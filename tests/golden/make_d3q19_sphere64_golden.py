"""Write the FP64 oracle's reference result for a 64^3 drop on a sphere after 1000 steps.

The workload (`workloads.sphere_drop_64`: the Sec. IV.C sphere of the 256^3 workload scaled by 1/4,
R = 10, with a tangent drop of radius 16, Carnahan-Starling EOS at 0.7 Tc, IVD walls with kappa = 0.2,
i.e. phi = 1.2 of Eq. 16, seeded 1e-6 density noise) is run for 1000 steps by the oracle alone
(`oracle.lbm`), and the density field, mass, density extremes, maximum |u| and the contact angle
(`oracle.contact_angle`, sphere fit) are stored in `d3q19_sphere64_1000.npz` beside this script.
After 1000 steps the drop is still spreading (about 86 degrees, falling); 64 nodes is the narrowest
grid whose columns the default FP32 D3Q19 step stages by TMA.  Nothing here touches the CUDA path.

Run from the repository root:  python tests/golden/make_d3q19_sphere64_golden.py   (about 15 minutes, one core)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import contact_angle as CA, eos as E, lbm  # noqa: E402

STEPS = 1000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "d3q19_sphere64_1000.npz")


def main():
    wl = W.sphere_drop_64(STEPS)
    N = wl.shape[0]
    eos = E.cs_config().at_reduced_temperature(wl.t_over_tc)
    g, l = E.maxwell(eos)
    mask = wl.mask()
    geo = lbm.Geometry(mask, "D3Q19")
    p = lbm.Params("D3Q19", eos, sigma=0.12, rho_l=l, rho_g=g, kappa=wl.kappa)
    f = lbm.init_state(wl.rho0(l, g), geo)
    t0 = time.time()
    done = 0
    while done < STEPS:
        n = min(100, STEPS - done)
        f = lbm.run(f, geo, p, n)
        done += n
        print(f"{done} steps, {time.time() - t0:.0f} s", flush=True)
    o, rho, u = lbm.observables(f, geo, p)
    np.savez_compressed(OUT, rho=rho, steps=STEPS, n=N)    # kept even if the fit below fails
    th, c, r, npts = CA.contact_angle(rho, mask, l, g, wl.drop_center, wl.body_center, wl.body_radius)
    np.savez_compressed(OUT, rho=rho, steps=STEPS, n=N, kappa=wl.kappa, rho_l=l, rho_g=g, mass=o.mass,
                        rho_max=o.rho_max, rho_min=o.rho_min, u_max=o.u_max, theta_deg=th,
                        drop_center=np.asarray(c), drop_radius=r, n_interface=npts)
    print(f"theta = {th:.4f} deg, r = {r:.4f}, mass = {o.mass:.12g}, wrote {OUT}")


if __name__ == "__main__":
    main()
