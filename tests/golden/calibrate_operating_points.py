"""Write paper_1812_06545_gb300/codes/operating_points.json: for every code of the mixed
family, the Eb/N0 at which the FP64 flooding sum-product oracle (max 20 iterations, early
exit) has a frame error rate of about 1e-2.

Calls only the oracle.  Method: FER on a 0.25 dB grid (2000 frames per point, seeded
frames), then log-linear interpolation of FER between the two grid points around 1e-2.

    python tests/golden/calibrate_operating_points.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1812_06545_gb300 import inputs as I  # noqa: E402

TARGET = 1e-2
FRAMES = 2000
OUT = os.path.join(ROOT, "paper_1812_06545_gb300", "codes", "operating_points.json")


def fer(code, name, eb, seed):
    _, _, c, L = I.make_frames(name, FRAMES, eb, seed, seed + 1)
    _, bits, _ = code.spa_flood(L, 20, early_exit=True)
    return float((bits != c).any(axis=1).mean())


def main():
    family = sorted(n for n in I.CODE_SPECS if n.endswith(tuple(f"_s{s}" for s in range(40, 52))))
    points = {}
    for name in family:
        mb, nb, Z, seed = I.CODE_SPECS[name]
        B, Zc = I.load_code(name)
        code = O.QCCode(B, Zc)
        rate = 1 - mb / nb
        eb = round((1.5 + 4.0 * (rate - 0.5)) * 4) / 4
        grid = []
        while True:
            f = fer(code, name, eb, 7000 + seed)
            grid.append((eb, f))
            print(f"{name}: {eb:.2f} dB FER {f:.4f}", flush=True)
            if f > TARGET and len(grid) == 1:
                eb += 0.25
                continue
            if f <= TARGET and len(grid) == 1:
                eb -= 0.25
                grid.sort()
                continue
            grid.sort()
            lo = [g for g in grid if g[1] > TARGET]
            hi = [g for g in grid if g[1] <= TARGET]
            if lo and hi:
                break
            eb = (grid[-1][0] + 0.25) if not hi else (grid[0][0] - 0.25)
        (e0, f0), (e1, f1) = lo[-1], hi[0]
        f1 = max(f1, 0.5 / FRAMES)
        x = e0 + (e1 - e0) * (np.log(TARGET) - np.log(f0)) / (np.log(f1) - np.log(f0))
        points[name] = {"ebn0_db": round(float(x), 3), "grid": [[e, f] for e, f in grid]}
    doc = {"what": "Eb/N0 per code at which the FP64 flooding sum-product oracle (max 20 iterations, early exit) "
                   "has a frame error rate of about 1e-2",
           "method": f"{FRAMES} seeded frames per 0.25 dB grid point, log-linear interpolation",
           "written_by": "tests/golden/calibrate_operating_points.py", "points": points}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
