"""Writes tests/golden/kbc_sphere_crop_128x64x64.npz: the FP64 oracle's
velocity after 1000 steps of the KBC D3Q27 flow past a sphere on the
128 x 64 x 64 crop, at a seeded uniform sample of fluid cells.

The crop is the full 512 x 256 x 256 channel scaled down by 4: sphere radius 8
centred at (32, 32, 32), Zou-He inlet u = (0.04, 0, 0) on x = 0, outflow on
x = 127, periodic in y and z, omega = 1.857, start f_0 = f^eq(1, u_in) on the
fluid-like cells.  The oracle takes about 1.4 s per step on one core, so the
1000-step result is stored rather than recomputed by the tests.

Run from the repository root:  python tests/golden/make_kbc_sphere_crop.py
It calls only the oracle and the seeded input generators.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lbm as O  # noqa: E402
from paper_2311_16080_gb300 import inputs as I  # noqa: E402

NX, NY, NZ = 128, 64, 64
RADIUS = 8
CENTER = (32, 32, 32)
U_IN = 0.04
OMEGA = 1.857
STEPS = 1000
N_SAMPLE = 16384
SEED = 1234
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kbc_sphere_crop_128x64x64.npz")


def setup():
    lat = O.Lattice(27)
    mask = I.sphere_channel_mask(NX, NY, NZ, radius=RADIUS, center=CENTER)
    rho = np.ones(mask.shape)
    u = np.zeros((3,) + mask.shape)
    u[0][O.fluid_like(mask)] = U_IN
    p = O.Params(lat, OMEGA, collision="kbc", bc=O.BC(3, inlet_u=(U_IN, 0.0, 0.0)))
    return lat, mask, rho, u, p


def sample_cells(mask):
    """Flat indices (x fastest) of N_SAMPLE distinct fluid-like cells."""
    fl = np.flatnonzero(O.fluid_like(mask).ravel())
    rng = np.random.default_rng(SEED)
    return np.sort(rng.choice(fl, size=N_SAMPLE, replace=False)).astype(np.int64)


def main():
    lat, mask, rho, u, p = setup()
    f = O.init_state(lat, rho, u, mask, p)
    t0 = time.time()
    for k in range(STEPS):
        f = O.step(lat, f, mask, p)
        if (k + 1) % 100 == 0:
            print(f"step {k + 1}  {time.time() - t0:.0f} s", flush=True)
    _, uu = O.macroscopic(lat, f, mask, p)
    idx = sample_cells(mask)
    u_s = uu.reshape(3, -1)[:, idx]
    u_fl = uu[:, O.fluid_like(mask)]
    np.savez_compressed(OUT, index=idx, u=u_s, steps=STEPS, omega=OMEGA, u_in=U_IN,
                        u_rms_all_fluid=float(np.sqrt((u_fl ** 2).sum() / u_fl.shape[1])))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
