"""Cases of the checked-build test (imported by tests/test_gpu_checked.py and run by it in
a child process against the bounds-checked library): every kernel path and job layout on
small and degenerate lattices, after one, two and three steps (both AA parities)."""
import sys

import numpy as np

from paper_2303_08163_gb300 import inputs

# (D, dims, precision, launch shape (kernel, threads[, stages, rows, seg, cap]), eq, bulk)
CASES = []
for prec in (0, 1, 2):
    CASES += [
        (2, (4, 4, 1), prec, (1, 128), 0, 0),          # tiny
        (3, (3, 5, 7), prec, (1, 128), 0, 0),          # odd sizes
        (3, (1, 1, 1), prec, (1, 32), 0, 0),           # every neighbour is the cell itself
        (3, (2, 2, 2), prec, (1, 32), 1, 1),           # N = 2 wraps
        (2, (1, 2, 1), prec, (1, 32), 2, 0),
        (2, (40, 18, 1), prec, (2, 256, 3, 4, 40, 2048), 0, 0),   # rows, y wrap
        (2, (40, 18, 1), prec, (2, 128, 2, 1, 16, 1024), 0, 1),   # segments + short last
        (3, (24, 10, 6), prec, (2, 128, 3, 3, 24, 1024), 1, 0),
        (3, (24, 10, 6), prec, (2, 256, 2, 1, 8, 1024), 0, 0),
    ]
CASES += [
    (3, (8, 1, 1), 2, (2, 128, 2, 1, 8, 1024), 0, 0),    # one 16-byte row, y and z wrap onto itself
    (3, (16, 2, 3), 2, (2, 128, 2, 2, 16, 1024), 2, 1),
    (3, (4, 3, 2), 1, (2, 128, 2, 3, 4, 1024), 0, 0),    # 16-byte FP32 rows
    (3, (2, 3, 2), 0, (2, 128, 2, 3, 2, 1024), 0, 0),    # 16-byte FP64 rows
    (3, (48, 6, 4), 2, (2, 256, 4, 6, 48, 1024), 0, 0),  # deeper pipeline, several rows
]


def run(lbm, out_path):
    """Run every case; save the stored state after 1, 2 and 3 steps (raw storage bits)."""
    res = {}
    for n, (D, dims, prec, shape, eq, bulk) in enumerate(CASES):
        rho, u = inputs.random_state(D, dims, seed=900 + n, u_max=0.1)
        lat = lbm.Lattice(lbm.D2Q9 if D == 2 else lbm.D3Q27, dims, 0.6, eq, bulk, prec)
        lat.set_launch_shape(*shape)
        lat.init_fields(rho, u)
        assert lat.launch_info()["kernel"] == shape[0], (n, lat.launch_info())
        for t in range(3):
            lat.step(1)
            lat.sync()
            res[f"case{n}_t{t + 1}"] = lat.get_populations("storage").view(np.uint8)
        lat.close()
    np.savez(out_path, **res)


if __name__ == "__main__":
    from paper_2303_08163_gb300 import lbm as _lbm
    _lbm.load()
    run(_lbm, sys.argv[1])
