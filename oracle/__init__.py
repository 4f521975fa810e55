"""CPU FP64 oracle of the pseudopotential MRT lattice Boltzmann step with the improved
virtual-density contact-angle scheme (Li, Yu & Luo, arXiv:1908.04443).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only the tests,
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may use it.  It shares no code
with the CUDA path (no tables, helpers or constants); the only common module is `workloads`,
which generates seeded inputs and holds none of the method's arithmetic.

The oracle is written to be checked by eye against the paper:

* `lattice`  - D2Q9 / D3Q19 velocities, weights, transformation matrices M, f^eq, Guo source G.
* `eos`      - Peng-Robinson (Eq. 18) and Carnahan-Starling pressures, psi (Eq. 6), the critical
               point and the Maxwell equal-area construction for the coexistence densities.
* `lbm`      - one time step in the paper's order: moments (Eq. 4), the improved virtual wall
               density (Eqs. 16-17), the interaction force (Eq. 5), the MRT collision with the
               consistency source (Eqs. 2, 7) and streaming with halfway bounce-back (Eq. 3, Fig. 3).
* `contact_angle` - interface extraction and a Kasa circle/sphere fit, giving theta on the body.

Everything is float64 and vectorised over nodes with numpy; per-node arithmetic follows the
equations term by term with no fusion or reordering beyond the equations themselves.
"""
