"""Write the FP64 oracle's statistics of a whole 800x800 frame to a golden file.

    python tests/golden/make_frame_stats.py frame800 0

Renders every pixel of scene `seed` of the named workload with the oracle
(only oracle/ and scenegen/ are used; about 20 minutes on 8 cores) and writes
tests/golden/<name>_seed<seed>_stats.txt with the frame's peak (max over
pixels and channels), its 99.9th percentile and its mean.  The BF16 parity
test takes the frame peak from this file, because its PSNR is defined with
the peak of the whole oracle image while the test samples pixels.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import scenegen  # noqa: E402
from oracle import render as orender  # noqa: E402


def main(name: str, seed: int) -> None:
    cfg = scenegen.CONFIGS[name]
    sc = scenegen.make_scene(cfg, seed)
    gb = scenegen.make_gbuffer(cfg.n_pixels, seed)
    prm = orender.Params.from_arrays(sc.table, sc.brdf, sc.irt, sc.env)
    opt = orender.Options.from_config(cfg)
    t0 = time.time()
    out = np.empty((cfg.n_pixels, 3))
    step = 8192
    for s in range(0, cfg.n_pixels, step):
        rows = np.arange(s, min(cfg.n_pixels, s + step))
        out[rows] = orender.render(gb, prm, opt, rows=rows)
        print(f"{s + rows.size}/{cfg.n_pixels} pixels, {time.time() - t0:.0f} s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_seed{seed}_stats.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 oracle over all {cfg.n_pixels} pixels of {name} seed {seed} "
                f"(tests/golden/make_frame_stats.py)\n")
        f.write(f"peak {out.max():.17g}\n")
        f.write(f"p999 {np.quantile(out, 0.999):.17g}\n")
        f.write(f"mean {out.mean():.17g}\n")
    print(path)


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]))
