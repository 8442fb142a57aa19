"""Write closed_forms.json: worked cases whose expected values follow from
the paper's equations in closed form (Sec. 3.1: the Beer-Lambert segment
opacity and the Riemann sum of Eq. 1 with front-to-back blending).

Each value is computed here from its formula with Python's `math`
(binary64), independently of the oracle and of the CUDA path; every input
is exact in binary32. Geometry common to every
case: a 33^3 vertex grid spans the unit cube [-1/2, 1/2]^3 (vertex spacing
h = 1/32); a step of 0.5 voxel is dt = 1/64 world units; a ray along -z that
enters the top face z = 1/2 crosses L = 1 and takes N = L/dt = 64 samples at
z_i = 1/2 - i dt, each weighted by the full dt.

    python tests/golden/make_golden.py
"""
import json
import math
import os

N_VERT = 33
STEP = 0.5
DT = STEP / (N_VERT - 1)          # 1/64
N = 64                            # L / dt for L = 1


def beer_lambert(sigma):
    # Sec. 3.1: alpha_i = 1 - exp(-dt tau); absorption-only (tau = d = sigma)
    # composited front to back gives 1 - A = prod (1 - alpha_i) = exp(-sigma N dt)
    return 1.0 - math.exp(-sigma * N * DT)


def constant_tf(rgb, tau):
    # Eq. 1 Riemann sum with premultiplied emission: C = sum_i T_i alpha_i rgb
    # = rgb (1 - exp(-tau N dt)), A = 1 - exp(-tau N dt)
    a = 1.0 - math.exp(-tau * N * DT)
    return [c * a for c in rgb] + [a]


def linear_ramp(d0, d1):
    # density linear in z: d(z) = d0 + (d1 - d0) (z + 1/2) (exact under
    # trilinear interpolation). Left Riemann sum from the entry face:
    # S = sum_{i<N} dt d(1/2 - i dt)
    s = sum(DT * (d0 + (d1 - d0) * (1.0 - i * DT)) for i in range(N))
    return s, 1.0 - math.exp(-s)


def main():
    ortho = {"width": 5, "height": 3, "ortho": True, "ortho_height": 0.5}
    cases = [
        {"id": "beer_lambert_ortho", "cite": "Sec. 3.1, Beer-Lambert segment opacity",
         "model": "absorption", "volume": {"kind": "constant", "value": 1.75}, "view": ortho,
         "eye": [0.0, 0.0, 2.0], "step": STEP, "pixels": "all", "N": N,
         "expected": [beer_lambert(1.75)]},
        {"id": "beer_lambert_perspective_centre", "cite": "Sec. 3.1, Beer-Lambert segment opacity",
         "model": "absorption", "volume": {"kind": "constant", "value": 1.75},
         "view": {"width": 5, "height": 5, "ortho": False}, "eye": [0.0, 0.0, 2.5], "step": STEP,
         "pixels": [12], "N": N, "expected": [beer_lambert(1.75)]},
        {"id": "constant_tf_emission_absorption", "cite": "Sec. 3.1, Eq. 1 and Eq. blend-forward",
         "model": "emission_absorption", "volume": {"kind": "constant", "value": 0.3},
         "tf": [[0.25, 0.5, 0.875, 6.0]] * 5, "view": ortho, "eye": [0.0, 0.0, 2.0], "step": STEP,
         "pixels": "all", "N": N, "expected": constant_tf([0.25, 0.5, 0.875], 6.0)},
    ]
    s, a = linear_ramp(0.25, 0.75)
    cases.append({"id": "linear_ramp_riemann_sum", "cite": "Sec. 3.1, Eq. 1 (Riemann sum from the entry face)",
                  "model": "absorption", "volume": {"kind": "ramp_z", "d0": 0.25, "d1": 0.75}, "view": ortho,
                  "eye": [0.0, 0.0, 2.0], "step": STEP, "pixels": "all", "N": N, "optical_depth": s,
                  "expected": [a]})
    out = {"grid": N_VERT, "note": "expected values from the closed forms in make_golden.py", "cases": cases}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
