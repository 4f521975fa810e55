"""Write the FP64 oracle's reference result for the 600 x 400 drop-on-cylinder workload.

The workload (Sec. IV.A geometry scaled up: cylinder R = 60 at (300, 150), drop r = 70 at (300, 280),
Carnahan-Starling EOS at 0.6 Tc, IVD walls with kappa = 0.15, i.e. phi = 1.15 of Eq. 16, seeded
1e-6 density noise) is run for its 20,000 steps by the oracle alone (`oracle.lbm`), and the density
field, mass, density extremes, maximum |u| and the contact angle (`oracle.contact_angle`) are stored
in `c2_600x400_kappa0.15_20000.npz` beside this script.  Nothing here touches the CUDA path.

Run from the repository root:  python tests/golden/make_c2_golden.py   (about 20 minutes, one core)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import contact_angle as CA, eos as E, lbm  # noqa: E402

KAPPA = 0.15
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_600x400_kappa0.15_20000.npz")


def main():
    wl = W.c2_cylinder_600x400(kappa=KAPPA)
    eos = E.cs_config().at_reduced_temperature(wl.t_over_tc)
    g, l = E.maxwell(eos)
    mask = wl.mask()
    geo = lbm.Geometry(mask, "D2Q9")
    p = lbm.Params("D2Q9", eos, sigma=0.12, rho_l=l, rho_g=g, kappa=KAPPA)
    f = lbm.init_state(wl.rho0(l, g), geo)
    t0 = time.time()
    done = 0
    while done < wl.steps:
        n = min(1000, wl.steps - done)
        f = lbm.run(f, geo, p, n)
        done += n
        print(f"{done} steps, {time.time() - t0:.0f} s", flush=True)
    o, rho, u = lbm.observables(f, geo, p)
    th, c, r, npts = CA.contact_angle(rho, mask, l, g, wl.drop_center, wl.body_center, wl.body_radius)
    np.savez_compressed(OUT, rho=rho, steps=wl.steps, kappa=KAPPA, rho_l=l, rho_g=g, mass=o.mass,
                        rho_max=o.rho_max, rho_min=o.rho_min, u_max=o.u_max, theta_deg=th,
                        drop_center=np.asarray(c), drop_radius=r, n_interface=npts)
    print(f"theta = {th:.4f} deg, r = {r:.4f}, mass = {o.mass:.12g}, wrote {OUT}")


if __name__ == "__main__":
    main()
